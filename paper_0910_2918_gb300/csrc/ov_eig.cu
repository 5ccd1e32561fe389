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
// A's spectrum gives spurious Ritz values near 0), then Rayleigh-Ritz with A on the leading
// m Ritz vectors of A^2 (the projected b x b and m x m eigenproblems are solved on the
// host, ov_small.cpp), residuals ||A x - lambda x||. At mu != 0 the left eigenvectors are the right eigenvectors of
// A^dag = gamma5 D_w(-mu) for conj(lambda): a second run with A^dag, matched by eigenvalue and
// biorthonormalised (L <- L (L^dag R)^{-dag}).
//
// All n-vectors are canonical complex doubles on the device; the matvecs run in the handle's
// arithmetic (ov_api.cu: apply_block).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <complex>
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
// the eigensolver: the m eigenpairs of smallest |lambda| of A (dagger = 0) or A^dag
// (dagger = 1) of lattice q, right eigenvectors into Rout ([m][n] device) and eigenvalues
// into lam (host); residuals (relative to ||A||) into res (host). Returns OV_OK or
// OV_NOT_CONVERGED (the best vectors are returned) or an error.
int eig_smallest(ov_handle* h, int q, int dagger, int m, int b, int deg, double tol, int maxit, double2* Rout,
                 std::vector<std::complex<double>>& lam, std::vector<double>& res, int* iters, int verbose) {
  using cd = std::complex<double>;
  cudaStream_t st = handle_stream(h);
  const size_t n = lattice_size(h, q);
  const bool herm = lattice_mu(h, q) == 0.0;
  // work: V (b), T0, T1 (b), W (b), Z (b) = 5 blocks; gram partials; small matrices
  const size_t blk = n * b;
  double2 *V = nullptr, *T0 = nullptr, *T1 = nullptr, *W = nullptr, *Z = nullptr, *part = nullptr, *G = nullptr;
  double* rpart = nullptr;
  double* rn = nullptr;
  auto cleanup = [&]() {
    for (void* p : {(void*)V, (void*)T0, (void*)T1, (void*)W, (void*)Z, (void*)part, (void*)G, (void*)rpart, (void*)rn})
      if (p) cudaFree(p);
  };
  const int rgrid = 64;
  if (cudaMalloc(&V, sizeof(double2) * blk) != cudaSuccess || cudaMalloc(&T0, sizeof(double2) * blk) != cudaSuccess ||
      cudaMalloc(&T1, sizeof(double2) * blk) != cudaSuccess || cudaMalloc(&W, sizeof(double2) * blk) != cudaSuccess ||
      cudaMalloc(&Z, sizeof(double2) * blk) != cudaSuccess ||
      cudaMalloc(&part, block_gram_part_bytes(b, b)) != cudaSuccess ||
      cudaMalloc(&G, sizeof(double2) * b * b * 2) != cudaSuccess ||
      cudaMalloc(&rpart, sizeof(double) * b * rgrid) != cudaSuccess || cudaMalloc(&rn, sizeof(double) * b) != cudaSuccess) {
    cleanup();
    return OV_ERR_NOMEM;
  }
  double2* Cd = G + b * b;  // small matrix upload
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
// inside the helper lambdas: report, the caller cleans up
#define LCK(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      fprintf(stderr, "libov: eigensolver: %s (%s:%d)\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return OV_ERR_CUDA;                                                           \
    }                                                                               \
  } while (0)
#define LRC(call)          \
  do {                     \
    int r_ = (call);       \
    if (r_ != OV_OK) return r_; \
  } while (0)
  std::vector<double2> Gh((size_t)b * b), Ch((size_t)b * b), wv(b), Sv((size_t)b * b);
  std::vector<double> wr(b);
  // random start (seeded per lattice; the result does not depend on it beyond roundoff)
  {
    std::vector<double2> r0(blk);
    unsigned s = 0x9e3779b9u ^ (unsigned)(q * 7919 + dagger);
    for (size_t e = 0; e < blk; ++e) {
      s ^= s << 13;
      s ^= s >> 17;
      s ^= s << 5;
      const double a = (s & 0xffffff) / 16777216.0 - 0.5;
      s ^= s << 13;
      s ^= s >> 17;
      s ^= s << 5;
      const double c = (s & 0xffffff) / 16777216.0 - 0.5;
      r0[e] = make_double2(a, c);
    }
    ECK(cudaMemcpyAsync(V, r0.data(), sizeof(double2) * blk, cudaMemcpyHostToDevice, st));
    ECK(cudaStreamSynchronize(st));
  }
  // orthonormalise the block X in place (Cholesky QR twice); Tmp: scratch block
  auto orth = [&](double2*& X, double2*& Tmp) -> int {
    for (int pass = 0; pass < 2; ++pass) {
      LCK(block_gram(n, X, n, b, X, n, b, part, G, st));
      LCK(cudaMemcpyAsync(Gh.data(), G, sizeof(double2) * b * b, cudaMemcpyDeviceToHost, st));
      LCK(cudaStreamSynchronize(st));
      double tr = 0.0;
      for (int i = 0; i < b; ++i) tr += Gh[(size_t)i * b + i].x;
      if (pass == 0)  // a tiny shift keeps the factorisation defined for a nearly dependent block
        for (int i = 0; i < b; ++i) Gh[(size_t)i * b + i].x += 1e-14 * tr;
      if (!small_chol_inv(b, Gh.data(), Ch.data())) return OV_ERR_BREAKDOWN;
      LCK(cudaMemcpyAsync(Cd, Ch.data(), sizeof(double2) * b * b, cudaMemcpyHostToDevice, st));
      LCK(block_mul(n, X, n, b, Cd, Tmp, n, b, 1.0, 0.0, st));
      std::swap(X, Tmp);
    }
    return OV_OK;
  };
  auto applyA2 = [&](const double2* X, double2* Y, double2* tmp) -> int {
    LRC(apply_block(h, q, b, X, tmp, dagger));
    LRC(apply_block(h, q, b, tmp, Y, dagger));
    return OV_OK;
  };
  RCK(orth(V, T0));
  // The filter needs an upper bound of |lambda|^2 over the whole spectrum: beyond it the
  // Chebyshev polynomial grows as fast as below the cut and would amplify the largest
  // eigenvectors. ||A||^2 from power steps on A^dag A (a lower estimate) with a 25% margin,
  // capped by the bound of the operator's form, ||A|| <= |m_w + 4| + 6 + 2 cosh(mu); a block
  // whose largest Ritz value comes near the bound enlarges it (safeguard below).
  double amax2 = 0.0;
  {
    ECK(cudaMemcpyAsync(T1, V, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
    for (int it = 0; it < 60; ++it) {
      RCK(apply_block(h, q, 1, T1, W, dagger));
      RCK(apply_block(h, q, 1, W, Z, 1 - dagger));
      ECK(block_gram(n, Z, n, 1, Z, n, 1, part, G, st));
      ECK(block_gram(n, T1, n, 1, Z, n, 1, part, G + 1, st));
      double2 g2[2];
      ECK(cudaMemcpyAsync(g2, G, sizeof(double2) * 2, cudaMemcpyDeviceToHost, st));
      ECK(cudaStreamSynchronize(st));
      amax2 = std::max(amax2, g2[1].x);  // Rayleigh quotient of A^dag A (T1 has unit norm)
      const double nz = sqrt(g2[0].x);
      double2 sc = make_double2(1.0 / nz, 0.0);
      ECK(cudaMemcpyAsync(Cd, &sc, sizeof(double2), cudaMemcpyHostToDevice, st));
      ECK(block_mul(n, Z, n, 1, Cd, T1, n, 1, 1.0, 0.0, st));
    }
    const double form = fabs(lattice_mass(h, q)) + 6.0 + 2.0 * cosh(lattice_mu(h, q));
    amax2 = std::min(1.25 * amax2, form * form);
  }
  const double anorm = sqrt(amax2);
  double a_cut = 0.05 * amax2;
  int it = 0;
  bool done = false;
  lam.assign(m, cd(0.0));
  res.assign(m, INFINITY);
  for (it = 1; it <= maxit && !done; ++it) {
    // filter: T_deg(l(A^2)) V, l(z) = s z + t maps [a_cut, amax2] onto [-1, 1]
    const double s = 2.0 / (amax2 - a_cut), t = -(amax2 + a_cut) / (amax2 - a_cut);
    // T0 = V, T1 = l(A^2) V, then T_{k+1} = 2 l(A^2) T_k - T_{k-1} (kept in V / T0 / T1)
    RCK(applyA2(V, W, Z));
    k_cheb<<<grid_n(blk), kEigThreads, 0, st>>>(blk, W, V, nullptr, s, t, 1, T1);
    ECK(cudaGetLastError());
    double2* Tm = V;   // T_{k-1}
    double2* Tc = T1;  // T_k
    double2* Tn = T0;  // T_{k+1}
    for (int k = 1; k < deg; ++k) {
      RCK(applyA2(Tc, W, Z));
      k_cheb<<<grid_n(blk), kEigThreads, 0, st>>>(blk, W, Tc, Tm, s, t, 0, Tn);
      ECK(cudaGetLastError());
      double2* o = Tm;
      Tm = Tc;
      Tc = Tn;
      Tn = o;
    }
    // the filtered block is Tc; make it V (the buffers are interchangeable)
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
    int orc = orth(V, T0);
    if (orc != OV_OK) {
      cleanup();
      return orc;
    }
    // Rayleigh-Ritz with A^2 on the block (its wanted eigenvalues are at the bottom of the
    // spectrum of A^2, so no spurious Ritz values; Rayleigh-Ritz with A on a subspace aimed
    // at the interior of A's spectrum gives spurious values near 0 from mixed +-lambda
    // vectors): Z = A V, Y = A Z, H2 = V^dag Y
    RCK(apply_block(h, q, b, V, Z, dagger));
    RCK(apply_block(h, q, b, Z, W, dagger));
    ECK(block_gram(n, V, n, b, W, n, b, part, G, st));
    ECK(cudaMemcpyAsync(Gh.data(), G, sizeof(double2) * b * b, cudaMemcpyDeviceToHost, st));
    ECK(cudaStreamSynchronize(st));
    bool ok;
    if (herm) {
      for (int i = 0; i < b; ++i)
        for (int j = 0; j < i; ++j) {  // symmetrise the projection (roundoff)
          const double2 u = Gh[(size_t)i * b + j], v = Gh[(size_t)j * b + i];
          const double2 avg = make_double2(0.5 * (u.x + v.x), 0.5 * (u.y - v.y));
          Gh[(size_t)i * b + j] = avg;
          Gh[(size_t)j * b + i] = make_double2(avg.x, -avg.y);
        }
      ok = small_eigh(b, Gh.data(), wr.data(), Sv.data());
      for (int i = 0; i < b; ++i) wv[i] = make_double2(wr[i], 0.0);
    } else {
      ok = small_eig(b, Gh.data(), wv.data(), Sv.data());
    }
    if (!ok) {
      cleanup();
      return OV_ERR_BREAKDOWN;
    }
    auto mag2 = [](double2 z) { return z.x * z.x + z.y * z.y; };
    std::vector<int> idx(b);
    for (int i = 0; i < b; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return mag2(wv[x]) < mag2(wv[y]); });
    for (int i = 0; i < b; ++i)
      for (int j = 0; j < b; ++j) Ch[(size_t)i * b + j] = Sv[(size_t)i * b + idx[j]];
    const double t2 = sqrt(mag2(wv[idx[b - 1]]));  // largest |theta^2| of the block
    // the Ritz vectors of A^2, orthonormalised again (the eigenvectors of a non-Hermitian
    // H2 are not orthogonal)
    ECK(cudaMemcpyAsync(Cd, Ch.data(), sizeof(double2) * b * b, cudaMemcpyHostToDevice, st));
    ECK(block_mul(n, V, n, b, Cd, T0, n, b, 1.0, 0.0, st));
    std::swap(V, T0);
    orc = orth(V, T0);
    if (orc != OV_OK) {
      cleanup();
      return orc;
    }
    // Rayleigh-Ritz with A on the leading m vectors: H1 = V_m^dag A V_m
    RCK(apply_block(h, q, m, V, Z, dagger));
    ECK(block_gram(n, V, n, m, Z, n, m, part, G, st));
    std::vector<double2> H1((size_t)m * m), S1((size_t)m * m), w1(m);
    std::vector<double> w1r(m);
    ECK(cudaMemcpyAsync(H1.data(), G, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, st));
    ECK(cudaStreamSynchronize(st));
    if (herm) {
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < i; ++j) {
          const double2 u = H1[(size_t)i * m + j], v = H1[(size_t)j * m + i];
          const double2 avg = make_double2(0.5 * (u.x + v.x), 0.5 * (u.y - v.y));
          H1[(size_t)i * m + j] = avg;
          H1[(size_t)j * m + i] = make_double2(avg.x, -avg.y);
        }
      ok = small_eigh(m, H1.data(), w1r.data(), S1.data());
      for (int i = 0; i < m; ++i) w1[i] = make_double2(w1r[i], 0.0);
    } else {
      ok = small_eig(m, H1.data(), w1.data(), S1.data());
    }
    if (!ok) {
      cleanup();
      return OV_ERR_BREAKDOWN;
    }
    std::vector<int> o1(m);
    for (int i = 0; i < m; ++i) o1[i] = i;
    std::sort(o1.begin(), o1.end(), [&](int x, int y) { return mag2(w1[x]) < mag2(w1[y]); });
    std::vector<double2> C1((size_t)m * m), th(m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) C1[(size_t)i * m + j] = S1[(size_t)i * m + o1[j]];
    for (int j = 0; j < m; ++j) th[j] = w1[o1[j]];
    // eigenvector estimates X = V_m C1 (in T1), A X = Z_m C1 (in W)
    ECK(cudaMemcpyAsync(Cd, C1.data(), sizeof(double2) * m * m, cudaMemcpyHostToDevice, st));
    ECK(block_mul(n, V, n, m, Cd, T1, n, m, 1.0, 0.0, st));
    ECK(block_mul(n, Z, n, m, Cd, W, n, m, 1.0, 0.0, st));
    // residuals ||A x_i - lambda_i x_i|| (x_i of unit norm)
    ECK(cudaMemcpyAsync(G, th.data(), sizeof(double2) * m, cudaMemcpyHostToDevice, st));
    k_resid_part<<<dim3(rgrid, m), kEigThreads, 0, st>>>(n, W, T1, n, G, rpart);
    k_resid_fin<<<(m + 127) / 128, 128, 0, st>>>(m, rgrid, rpart, rn);
    ECK(cudaGetLastError());
    std::vector<double> r(m);
    ECK(cudaMemcpyAsync(r.data(), rn, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    ECK(cudaStreamSynchronize(st));
    double worst = 0.0;
    for (int i = 0; i < m; ++i) {
      lam[i] = cd(th[i].x, th[i].y);
      res[i] = r[i] / anorm;
      worst = std::max(worst, res[i]);
    }
    if (verbose)
      fprintf(stderr, "{\"ov_eig\": %d, \"dagger\": %d, \"worst_residual\": %.3e, \"lambda_m\": %.6f, \"cut\": %.6f}\n",
              it, dagger, worst, std::abs(lam[m - 1]), sqrt(a_cut));
    done = worst <= tol;
    if (done) ECK(cudaMemcpyAsync(Rout, T1, sizeof(double2) * n * m, cudaMemcpyDeviceToDevice, st));
    // next filter interval: damp everything beyond the block's largest Ritz value of A^2; one
    // in the upper half of [0, bound] means vectors from the top of the spectrum were
    // amplified: widen the bound and start the interval afresh
    if (t2 > 0.5 * amax2) {
      amax2 = std::max(2.0 * amax2, 1.25 * t2);
      a_cut = 0.05 * amax2;
    } else {
      a_cut = std::min(std::max(t2, 1e-6 * amax2), 0.9 * amax2);
    }
  }
  if (!done) ECK(cudaMemcpyAsync(Rout, T1, sizeof(double2) * n * m, cudaMemcpyDeviceToDevice, st));
  if (iters) *iters = it - 1;
  ECK(cudaStreamSynchronize(st));
  cleanup();
#undef ECK
#undef RCK
#undef LCK
#undef LRC
  return done ? OV_OK : OV_NOT_CONVERGED;
}

}  // namespace ov
