// Roberts-Higham sign of dense matrices for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: applications that reserve all device memory up
// front for their own pool (a lattice code's field allocator, a framework's caching
// allocator), where an allocation by the library fails or fragments the pool, and code
// that must not pay the implicit device synchronisation cudaMalloc/cudaFree can impose.
// ov_rh_sign_noalloc serves them: the caller passes device buffers for the input and the
// output, the iterate S_n lives in the output buffer, and the only other scratch (pivot
// rows and per-matrix flags) is the file-scope array below, which every GPU that loads
// the library holds until the process exits.
#include <math.h>
#include <mutex>

#include <algorithm>

#include "ov_internal.h"
#include "ov_types.cuh"

namespace ov {
namespace {

constexpr int kNoAllocMaxCount = 64;  // matrices per call
constexpr int kNoAllocThreads = 1024;
// dynamic shared memory of one CTA: the m x m working matrix plus the column / reduction
// buffer; at m = kMaxL it must fit the 227 KB a CTA may opt in to on sm_100-class GPUs
constexpr size_t noalloc_smem(int m) {
  return (size_t)m * m * sizeof(double2) + ((size_t)m * sizeof(double2) > 512 ? (size_t)m * sizeof(double2) : 512);
}
static_assert(noalloc_smem(kMaxL) <= 232448, "working matrix of the largest size exceeds 227 KB of shared memory");

struct NoAllocScratch {
  int perm[kNoAllocMaxCount][kMaxL];  // row interchanges of the current inversion
  int ok[kNoAllocMaxCount];           // 1 converged, 0 not
  int its[kNoAllocMaxCount];          // iterations used
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// device address of g_noalloc_scratch per device (the host-side name is only a stand-in)
constexpr int kMaxDevices = 64;
NoAllocScratch* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

__device__ __forceinline__ double2 na_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 na_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double na_abs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 na_inv(double2 b) {
  const double s = fmax(fabs(b.x), fabs(b.y));
  if (s == 0.0) return make_double2(INFINITY, INFINITY);
  const double2 bs = make_double2(b.x / s, b.y / s);
  const double d = bs.x * bs.x + bs.y * bs.y;
  return make_double2(bs.x / (d * s), -bs.y / (d * s));
}

// One CTA per matrix: S_0 = T, S_{n+1} = (S_n + S_n^{-1})/2 (Eq. (Roberts)), with the
// inverse by in-place Gauss-Jordan elimination with partial pivoting in shared memory.
__global__ void __launch_bounds__(kNoAllocThreads) k_rh_noalloc(int m, const double2* __restrict__ T, double2* S,
                                                                NoAllocScratch* scr, double rh_tol, int rh_maxit) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int mid = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  double2* W = (double2*)smem;
  double2* col = W + (size_t)m * m;  // column buffer, reduction scratch, pivot slot
  double* red = (double*)col;
  int* piv_slot = (int*)col;
  double2* Sg = S + (size_t)mid * m * m;  // iterate in the caller's output buffer
  int* perm = scr->perm[mid];
  for (int e = tid; e < m * m; e += nth) Sg[e] = T[(size_t)mid * m * m + e];
  __syncthreads();
  int ok = 0, it = 0;
  for (it = 1; it <= rh_maxit; ++it) {
    for (int e = tid; e < m * m; e += nth) W[e] = Sg[e];
    __syncthreads();
    bool singular = false;
    for (int j = 0; j < m; ++j) {
      if (tid < 32) {
        double best = -1.0;
        int bi = j;
        for (int i = j + tid; i < m; i += 32) {
          const double a2 = na_abs2(W[(size_t)i * m + j]);
          if (a2 > best) { best = a2; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (tid == 0) piv_slot[0] = best > 0.0 ? bi : -1;
      }
      __syncthreads();
      const int p = piv_slot[0];
      __syncthreads();
      if (p < 0) { singular = true; break; }
      if (p != j)
        for (int c = tid; c < m; c += nth) {
          const double2 t = W[(size_t)j * m + c];
          W[(size_t)j * m + c] = W[(size_t)p * m + c];
          W[(size_t)p * m + c] = t;
        }
      if (tid == 0) perm[j] = p;
      __syncthreads();
      const double2 inv = na_inv(W[(size_t)j * m + j]);
      __syncthreads();
      for (int c = tid; c < m; c += nth) W[(size_t)j * m + c] = c == j ? inv : na_mul(W[(size_t)j * m + c], inv);
      for (int i = tid; i < m; i += nth) col[i] = i == j ? make_double2(0.0, 0.0) : W[(size_t)i * m + j];
      __syncthreads();
      for (int i = tid; i < m; i += nth)
        if (i != j) W[(size_t)i * m + j] = make_double2(0.0, 0.0);
      __syncthreads();
      for (int e = tid; e < m * m; e += nth) {
        const int i = e / m;
        if (i == j) continue;
        const int c = e - i * m;
        W[e] = na_sub(W[e], na_mul(col[i], W[(size_t)j * m + c]));
      }
      __syncthreads();
    }
    if (singular) { ok = 0; break; }
    for (int j = m - 1; j >= 0; --j) {
      const int p = perm[j];
      if (p != j)
        for (int i = tid; i < m; i += nth) {
          const double2 t = W[(size_t)i * m + j];
          W[(size_t)i * m + j] = W[(size_t)i * m + p];
          W[(size_t)i * m + p] = t;
        }
      __syncthreads();
    }
    double dif = 0.0, nrm = 0.0;
    bool fin = true;
    for (int e = tid; e < m * m; e += nth) {
      const double2 sn = Sg[e];
      const double2 s1 = make_double2(0.5 * (sn.x + W[e].x), 0.5 * (sn.y + W[e].y));
      fin = fin && isfinite(s1.x) && isfinite(s1.y);
      dif += na_abs2(na_sub(s1, sn));
      nrm += na_abs2(s1);
      Sg[e] = s1;
    }
    __syncthreads();
    dif = warp_sum(dif);
    nrm = warp_sum(nrm);
    const int fin_all = __syncthreads_and(fin ? 1 : 0);
    if ((tid & 31) == 0) { red[(tid >> 5) * 2] = dif; red[(tid >> 5) * 2 + 1] = nrm; }
    __syncthreads();
    double D = 0.0, N = 0.0;
    for (int q = 0; q < (nth >> 5); ++q) { D += red[2 * q]; N += red[2 * q + 1]; }
    __syncthreads();
    if (!fin_all || !isfinite(D) || !isfinite(N)) { ok = 0; break; }
    if (sqrt(D) <= rh_tol * sqrt(N)) { ok = 1; break; }
  }
  if (tid == 0) {
    scr->ok[mid] = ok;
    scr->its[mid] = it > rh_maxit ? rh_maxit : it;
  }
}

// Set-up once per device, with that device current: the device address of the
// scratch array (cudaGetSymbolAddress). Returns nullptr on failure.
NoAllocScratch* scratch_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) return nullptr;
    g_scratch_addr[dev] = (NoAllocScratch*)ptr;
  }
  return g_scratch_addr[dev];
}

}  // namespace
}  // namespace ov

using namespace ov;

extern "C" int ov_rh_sign_noalloc(int count, int m, const void* T, void* S, int* iters, double rh_tol, int rh_maxit,
                                  void* stream) {
  if (count < 1 || m < 1 || !T || !S || !(rh_tol > 0.0) || rh_maxit < 1) return OV_ERR_ARG;
  if (count > kNoAllocMaxCount || m > kMaxL) return OV_ERR_TOO_LARGE;
  NoAllocScratch* scr = scratch_for_current_device();
  if (!scr) return OV_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = noalloc_smem(m);
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return OV_ERR_CUDA;
  if (smem > (size_t)optin) return OV_ERR_TOO_LARGE;
  if (cudaFuncSetAttribute(k_rh_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return OV_ERR_CUDA;
  k_rh_noalloc<<<count, kNoAllocThreads, smem, st>>>(m, (const double2*)T, (double2*)S, scr, rh_tol, rh_maxit);
  if (cudaGetLastError() != cudaSuccess) return OV_ERR_CUDA;
  int ok[kNoAllocMaxCount], its[kNoAllocMaxCount];
  if (cudaMemcpyAsync(ok, scr->ok, sizeof(int) * count, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(its, scr->its, sizeof(int) * count, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return OV_ERR_CUDA;
  int rc = OV_OK;
  for (int i = 0; i < count; ++i) {
    if (iters) iters[i] = its[i];
    if (!ok[i]) rc = OV_ERR_RH_NOCONV;
  }
  return rc;
}
