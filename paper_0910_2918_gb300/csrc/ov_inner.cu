// Inner level of the nested method, in double precision (Sec. 3, Eqs. (nested),
// (precond); Sec. 2, Eq. (Roberts)).
//
//  k_inner   one CTA per problem: tridiagonal LU with partial pivoting of the Ritz
//            matrix H_k (row interchanges between neighbouring rows only), then l steps
//            of Lanczos (mu = 0) or two-sided Lanczos (mu != 0) on M = H_k + H_k^{-1}
//            from e_1. M u = H u + H^{-1} u and M^dag w = H^dag w + H^{-dag} w both use
//            the one factorisation (the solve with H^dag runs the factors backwards).
//  k_rh      one CTA per matrix: Roberts-Higham S_{n+1} = (S_n + S_n^{-1})/2 with an
//            in-place Gauss-Jordan inversion (partial pivoting) of the whole l x l
//            matrix in shared memory (l <= 120 complex: 225 KB).
//  k_combine one CTA per problem: c = Q_l s, the inner estimate against the leading
//            (l - dl) block, the outer estimate against the previous check.
#include <math.h>

#include <algorithm>

#include "ov_internal.h"
#include "ov_types.cuh"

namespace ov {

constexpr int kInnerThreads = 256;

__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  // scaled to avoid overflow of |b|^2 for large |b|
  double s = fmax(fabs(b.x), fabs(b.y));
  if (s == 0.0) return make_double2(INFINITY, INFINITY);
  double2 bs = make_double2(b.x / s, b.y / s), as = make_double2(a.x / s, a.y / s);
  double d = bs.x * bs.x + bs.y * bs.y;
  return make_double2((as.x * bs.x + as.y * bs.y) / d, (as.y * bs.x - as.x * bs.y) / d);
}
__device__ __forceinline__ double2 zinv(double2 b) { return zdiv(make_double2(1.0, 0.0), b); }

// block sum over kInnerThreads threads; result returned to every thread
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

struct InnerSmem {
  double2 *d, *a, *c;           // H diagonal, subdiagonal (row m, col m-1), superdiagonal (row m, col m+1)
  double2 *uinv, *u1, *u2, *l;  // LU factors
  unsigned char* sw;            // row interchange at step m
  double2 *q, *qp, *w, *wp, *u, *z;
  double* red;
};

// x = H^{-1} b with the GEPP factors (x may alias nothing; y is scratch of size k)
__device__ void tri_solve(const InnerSmem& S, int k, const double2* b, double2* x) {
  double2 cur = b[0];
  for (int m = 0; m < k - 1; ++m) {
    const double2 nb = b[m + 1];
    if (!S.sw[m]) {
      x[m] = cur;
      cur = zsub(nb, zmul(S.l[m], cur));
    } else {
      x[m] = nb;
      cur = zsub(cur, zmul(S.l[m], nb));
    }
  }
  x[k - 1] = cur;
  x[k - 1] = zmul(x[k - 1], S.uinv[k - 1]);
  if (k >= 2) x[k - 2] = zmul(zsub(x[k - 2], zmul(S.u1[k - 2], x[k - 1])), S.uinv[k - 2]);
  for (int m = k - 3; m >= 0; --m)
    x[m] = zmul(zsub(zsub(x[m], zmul(S.u1[m], x[m + 1])), zmul(S.u2[m], x[m + 2])), S.uinv[m]);
}

// z = H^{-dag} b: H = E^{-1} U with E the product of the elimination steps, so
// H^dag z = b  <=>  U^dag g = b, z = E_1^dag ... E_{k-1}^dag g.
__device__ void tri_solve_dag(const InnerSmem& S, int k, const double2* b, double2* z) {
  for (int m = 0; m < k; ++m) {
    double2 t = b[m];
    if (m >= 1) t = zsub(t, zmul(zconj(S.u1[m - 1]), z[m - 1]));
    if (m >= 2) t = zsub(t, zmul(zconj(S.u2[m - 2]), z[m - 2]));
    z[m] = zmul(t, zconj(S.uinv[m]));
  }
  for (int m = k - 2; m >= 0; --m) {
    const double2 cl = zconj(S.l[m]);
    const double2 gi = z[m], gn = z[m + 1];
    if (!S.sw[m]) {
      z[m] = zsub(gi, zmul(cl, gn));
    } else {
      z[m] = gn;
      z[m + 1] = zsub(gi, zmul(cl, gn));
    }
  }
}

// LU with partial pivoting of the tridiagonal H (thread 0). Returns false if singular.
__device__ bool tri_factor(const InnerSmem& S, int k) {
  double2 dd = S.d[0];
  double2 ee = k > 1 ? S.c[0] : make_double2(0.0, 0.0);
  for (int m = 0; m < k - 1; ++m) {
    const double2 an = S.a[m + 1], dn = S.d[m + 1];
    const double2 cn = (m + 1 <= k - 2) ? S.c[m + 1] : make_double2(0.0, 0.0);
    double2 r0, r1, r2, lm;
    if (zabs2(dd) >= zabs2(an)) {
      if (zabs2(dd) == 0.0) return false;
      lm = zdiv(an, dd);
      r0 = dd; r1 = ee; r2 = make_double2(0.0, 0.0);
      dd = zsub(dn, zmul(lm, ee));
      ee = cn;
      S.sw[m] = 0;
    } else {
      lm = zdiv(dd, an);
      r0 = an; r1 = dn; r2 = cn;
      dd = zsub(ee, zmul(lm, dn));
      ee = zscale(zmul(lm, cn), -1.0);
      S.sw[m] = 1;
    }
    S.uinv[m] = zinv(r0);
    S.u1[m] = r1;
    S.u2[m] = r2;
    S.l[m] = lm;
  }
  if (zabs2(dd) == 0.0) return false;
  S.uinv[k - 1] = zinv(dd);
  return true;
}

// y = H x (parallel)
__device__ __forceinline__ void tri_mul(const InnerSmem& S, int k, const double2* x, double2* y, bool dag) {
  for (int m = threadIdx.x; m < k; m += blockDim.x) {
    double2 t;
    if (!dag) {
      t = zmul(S.d[m], x[m]);
      if (m >= 1) t = zadd(t, zmul(S.a[m], x[m - 1]));
      if (m + 1 < k) t = zadd(t, zmul(S.c[m], x[m + 1]));
    } else {
      // (H^dag)_{m,m} = conj d_m, (H^dag)_{m,m-1} = conj H_{m-1,m} = conj c_{m-1},
      // (H^dag)_{m,m+1} = conj H_{m+1,m} = conj a_{m+1}
      t = zmul(zconj(S.d[m]), x[m]);
      if (m >= 1) t = zadd(t, zmul(zconj(S.c[m - 1]), x[m - 1]));
      if (m + 1 < k) t = zadd(t, zmul(zconj(S.a[m + 1]), x[m + 1]));
    }
    y[m] = t;
  }
}

__global__ void __launch_bounds__(kInnerThreads) k_inner(const int* __restrict__ k_dev, const int* __restrict__ l_dev,
                                                         int hermitian, const double2* __restrict__ alp,
                                                         const double2* __restrict__ bet,
                                                         const double2* __restrict__ gam, int ldc, InnerWork w) {
  int* fail = w.fail;
  extern __shared__ __align__(16) unsigned char smem[];
  const int prob = blockIdx.x;
  const int k = k_dev[prob];
  const int l = min(l_dev[prob], k);
  const int tid = threadIdx.x;
  InnerSmem S;
  {
    double2* base = (double2*)smem;
    S.d = base; S.a = base + k; S.c = base + 2 * k;
    S.uinv = base + 3 * k; S.u1 = base + 4 * k; S.u2 = base + 5 * k; S.l = base + 6 * k;
    S.q = base + 7 * k; S.qp = base + 8 * k; S.w = base + 9 * k; S.wp = base + 10 * k;
    S.u = base + 11 * k; S.z = base + 12 * k;
    S.red = (double*)(base + 13 * k);
    S.sw = (unsigned char*)(S.red + 32);
  }
  const double2* al = alp + (size_t)prob * ldc;
  const double2* be = bet + (size_t)prob * ldc;
  const double2* ga = gam + (size_t)prob * ldc;
  for (int m = tid; m < k; m += blockDim.x) {
    double2 dm = al[m + 1];
    double2 am = m >= 1 ? be[m + 1] : make_double2(0.0, 0.0);
    double2 cm = m + 1 < k ? ga[m + 2] : make_double2(0.0, 0.0);
    if (hermitian) { dm.y = 0.0; am.y = 0.0; cm = m + 1 < k ? make_double2(be[m + 2].x, 0.0) : cm; }
    S.d[m] = dm; S.a[m] = am; S.c[m] = cm;
    const double2 zero = make_double2(0.0, 0.0);
    S.q[m] = m == 0 ? make_double2(1.0, 0.0) : zero;
    S.w[m] = S.q[m];
    S.qp[m] = zero; S.wp[m] = zero;
  }
  __syncthreads();
  __shared__ int s_ok;
  if (tid == 0) s_ok = tri_factor(S, k) ? 1 : 0;
  __syncthreads();
  if (!s_ok) {
    if (tid == 0) { fail[prob] = 1; w.leff[prob] = 0; }
    return;
  }
  double2* Q = w.Q + (size_t)prob * w.ld * kMaxL;
  double2* T = w.T + (size_t)prob * kMaxL * 3;
  double2 b_i = make_double2(0.0, 0.0), g_i = make_double2(0.0, 0.0);  // inner beta_i, gamma_i
  int done = 0;
  const double exhaust_tol = 1e-13;
  for (int i = 0; i < l; ++i) {
    for (int m = tid; m < k; m += blockDim.x) Q[(size_t)m * kMaxL + i] = S.q[m];
    // u = M q = H q + H^{-1} q ; z = M^dag w (two-sided)
    if (tid == 0) tri_solve(S, k, S.q, S.u);
    if (!hermitian && tid == 32) tri_solve_dag(S, k, S.w, S.z);
    __syncthreads();
    double mq2 = 0.0;
    for (int m = tid; m < k; m += blockDim.x) {
      double2 t = zmul(S.d[m], S.q[m]);
      if (m >= 1) t = zadd(t, zmul(S.a[m], S.q[m - 1]));
      if (m + 1 < k) t = zadd(t, zmul(S.c[m], S.q[m + 1]));
      t = zadd(t, S.u[m]);
      mq2 += zabs2(t);
      S.u[m] = zsub(t, hermitian ? zscale(S.qp[m], b_i.x) : zmul(g_i, S.qp[m]));  // p
      if (!hermitian) {
        double2 y = zmul(zconj(S.d[m]), S.w[m]);
        if (m >= 1) y = zadd(y, zmul(zconj(S.c[m - 1]), S.w[m - 1]));
        if (m + 1 < k) y = zadd(y, zmul(zconj(S.a[m + 1]), S.w[m + 1]));
        y = zadd(y, S.z[m]);
        S.z[m] = zsub(y, zmul(zconj(b_i), S.wp[m]));  // r
      }
    }
    __syncthreads();
    // alpha = w^dag p (q^dag p in the Hermitian case)
    double are = 0.0, aim = 0.0;
    for (int m = tid; m < k; m += blockDim.x) {
      const double2 wm = hermitian ? S.q[m] : S.w[m];
      const double2 pm = S.u[m];
      are += wm.x * pm.x + wm.y * pm.y;
      aim += wm.x * pm.y - wm.y * pm.x;
    }
    are = block_sum(are, S.red);
    aim = hermitian ? 0.0 : block_sum(aim, S.red);
    const double mqn = sqrt(block_sum(mq2, S.red));
    const double2 a_i = make_double2(are, aim);
    if (tid == 0) T[i * 3 + 0] = a_i;
    done = i + 1;
    if (i == l - 1) break;
    // q~ = p - alpha q ; w~ = r - conj(alpha) w ; delta
    double dre = 0.0, dim = 0.0, n2 = 0.0;
    for (int m = tid; m < k; m += blockDim.x) {
      const double2 qt = zsub(S.u[m], zmul(a_i, S.q[m]));
      S.u[m] = qt;
      if (hermitian) {
        n2 += zabs2(qt);
      } else {
        const double2 wt = zsub(S.z[m], zmul(zconj(a_i), S.w[m]));
        S.z[m] = wt;
        dre += wt.x * qt.x + wt.y * qt.y;
        dim += wt.x * qt.y - wt.y * qt.x;
      }
    }
    double bn;
    double2 gn;
    if (hermitian) {
      bn = sqrt(block_sum(n2, S.red));
      gn = make_double2(bn, 0.0);
    } else {
      dre = block_sum(dre, S.red);
      dim = block_sum(dim, S.red);
      const double ad = sqrt(dre * dre + dim * dim);
      bn = sqrt(ad);
      gn = bn > 0.0 ? make_double2(dre / bn, dim / bn) : make_double2(0.0, 0.0);
    }
    if (!(bn > exhaust_tol * mqn)) break;  // inner space exhausted: T_i is exact
    if (tid == 0) {
      T[(i + 1) * 3 + 1] = make_double2(bn, 0.0);
      T[(i + 1) * 3 + 2] = gn;
    }
    const double2 wdiv = zinv(zconj(gn));
    __syncthreads();
    for (int m = tid; m < k; m += blockDim.x) {
      S.qp[m] = S.q[m];
      S.q[m] = zscale(S.u[m], 1.0 / bn);
      if (!hermitian) {
        S.wp[m] = S.w[m];
        S.w[m] = zmul(S.z[m], wdiv);
      }
    }
    b_i = make_double2(bn, 0.0);
    g_i = gn;
    __syncthreads();
  }
  if (tid == 0) {
    w.leff[prob] = done;
    T[0 * 3 + 1] = make_double2(0.0, 0.0);
    T[0 * 3 + 2] = make_double2(0.0, 0.0);
    fail[prob] = 0;
  }
}

// ------------------------------------------------------------ Roberts-Higham
// CTA `m2` handles matrix m2: problems [0, count) are T_{leff}, [count, 2 count) are
// T_{leff - dl} (the inner estimate); dense mode reads full matrices.
template <bool CPLX>
struct RhElem;
template <> struct RhElem<true> { using T = double2; };
template <> struct RhElem<false> { using T = double; };

__device__ __forceinline__ double2 rz(double2 a) { return a; }
__device__ __forceinline__ double el_abs2(double a) { return a * a; }
__device__ __forceinline__ double el_abs2(double2 a) { return zabs2(a); }
__device__ __forceinline__ double el_mul(double a, double b) { return a * b; }
__device__ __forceinline__ double2 el_mul(double2 a, double2 b) { return zmul(a, b); }
__device__ __forceinline__ double el_sub(double a, double b) { return a - b; }
__device__ __forceinline__ double2 el_sub(double2 a, double2 b) { return zsub(a, b); }
__device__ __forceinline__ double el_inv(double a) { return 1.0 / a; }
__device__ __forceinline__ double2 el_inv(double2 a) { return zinv(a); }
__device__ __forceinline__ double el_avg(double a, double b) { return 0.5 * (a + b); }
__device__ __forceinline__ double2 el_avg(double2 a, double2 b) { return make_double2(0.5 * (a.x + b.x), 0.5 * (a.y + b.y)); }
__device__ __forceinline__ double el_from(double2 a) { return a.x; }
__device__ __forceinline__ double2 el_from2(double2 a) { return a; }
__device__ __forceinline__ double2 el_to2(double a) { return make_double2(a, 0.0); }
__device__ __forceinline__ double2 el_to2(double2 a) { return a; }
__device__ __forceinline__ double el_zero(double) { return 0.0; }
__device__ __forceinline__ double2 el_zero(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double el_one(double) { return 1.0; }
__device__ __forceinline__ double2 el_one(double2) { return make_double2(1.0, 0.0); }
__device__ __forceinline__ bool el_finite(double a) { return isfinite(a); }
__device__ __forceinline__ bool el_finite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

template <class E>
__device__ __forceinline__ E el_load(const double2* p) {
  if constexpr (sizeof(E) == sizeof(double)) return p->x; else return *(const E*)p;
}

template <bool CPLX>
__global__ void __launch_bounds__(1024) k_rh(int count, int dense_m, const double2* __restrict__ dense_T,
                                             InnerWork w, int dl, double rh_tol, int rh_maxit, int mid0) {
  using E = typename RhElem<CPLX>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const int mid = mid0 + blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  int m;
  if (dense_m > 0) {
    m = dense_m;
  } else {
    const int prob = mid % count;
    const int le = w.leff[prob];
    m = mid < count ? le : le - dl;
  }
  if (m <= 0) {
    if (tid == 0) { w.rh_ok[mid] = m == 0 ? 0 : 1; w.rh_its[mid] = 0; }
    return;
  }
  E* W = (E*)smem;                    // m x m working matrix
  E* col = W + (size_t)m * m;         // column buffer / reduction scratch
  double* red = (double*)col;
  int* piv_slot = (int*)col;
  double2* Sg = w.S + (size_t)mid * kMaxL * kMaxL;  // global S_n (row-major, leading dim m)
  int* perm = w.perm + (size_t)mid * kMaxL;
  // S_0 = T
  for (int e = tid; e < m * m; e += nth) {
    const int i = e / m, j = e % m;
    double2 v = make_double2(0.0, 0.0);
    if (dense_m > 0) {
      v = dense_T[(size_t)mid * m * m + e];
    } else {
      const double2* T = w.T + (size_t)(mid % count) * kMaxL * 3;
      if (i == j) v = T[i * 3 + 0];
      else if (i == j + 1) v = T[i * 3 + 1];      // subdiagonal beta_{i}
      else if (j == i + 1) v = T[j * 3 + 2];      // superdiagonal gamma_{j}
    }
    if (!CPLX) v.y = 0.0;
    Sg[e] = v;
  }
  __syncthreads();
  int ok = 0, it = 0;
  for (it = 1; it <= rh_maxit; ++it) {
    for (int e = tid; e < m * m; e += nth) W[e] = el_load<E>(&Sg[e]);
    __syncthreads();
    bool singular = false;
    for (int j = 0; j < m; ++j) {
      // pivot search in column j (warp 0; ties keep the smaller row)
      if (tid < 32) {
        double best = -1.0;
        int bi = j;
        for (int i = j + tid; i < m; i += 32) {
          const double a2 = el_abs2(W[(size_t)i * m + j]);
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
          const E t = W[(size_t)j * m + c];
          W[(size_t)j * m + c] = W[(size_t)p * m + c];
          W[(size_t)p * m + c] = t;
        }
      if (tid == 0) perm[j] = p;
      __syncthreads();
      const E inv = el_inv(W[(size_t)j * m + j]);
      __syncthreads();
      for (int c = tid; c < m; c += nth) W[(size_t)j * m + c] = c == j ? inv : el_mul(W[(size_t)j * m + c], inv);
      for (int i = tid; i < m; i += nth) col[i] = i == j ? el_zero(inv) : W[(size_t)i * m + j];
      __syncthreads();
      for (int i = tid; i < m; i += nth)
        if (i != j) W[(size_t)i * m + j] = el_zero(inv);
      __syncthreads();
      {
        // 32 x 32 thread tile: thread (ty, tx) updates rows ty + 32a and columns tx + 32b,
        // holding its entries of the pivot row in registers (m <= 120 < 4 * 32)
        const int tx = tid & 31, ty = tid >> 5;
        E rowj[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int c = tx + 32 * b;
          rowj[b] = c < m ? W[(size_t)j * m + c] : el_zero(inv);
        }
        for (int i = ty; i < m; i += 32) {
          if (i == j) continue;
          const E f = col[i];
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int c = tx + 32 * b;
            if (c < m) W[(size_t)i * m + c] = el_sub(W[(size_t)i * m + c], el_mul(f, rowj[b]));
          }
        }
      }
      __syncthreads();
    }
    if (singular) { ok = 0; break; }
    // undo the row interchanges as column interchanges, last first
    for (int j = m - 1; j >= 0; --j) {
      const int p = perm[j];
      if (p != j)
        for (int i = tid; i < m; i += nth) {
          const E t = W[(size_t)i * m + j];
          W[(size_t)i * m + j] = W[(size_t)i * m + p];
          W[(size_t)i * m + p] = t;
        }
      __syncthreads();
    }
    // S_{n+1} = (S_n + S_n^{-1}) / 2 ; convergence test in the Frobenius norm
    double dif = 0.0, nrm = 0.0;
    bool fin = true;
    for (int e = tid; e < m * m; e += nth) {
      const E sn = el_load<E>(&Sg[e]);
      const E s1 = el_avg(sn, W[e]);
      fin = fin && el_finite(s1);
      dif += el_abs2(el_sub(s1, sn));
      nrm += el_abs2(s1);
      Sg[e] = el_to2(s1);
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
    w.rh_ok[mid] = ok;
    w.rh_its[mid] = it > rh_maxit ? rh_maxit : it;
  }
  for (int i = tid; i < m; i += nth) w.s[(size_t)mid * kMaxL + i] = Sg[(size_t)i * m];
}

// ------------------------------------------------- Roberts-Higham in double-float
// The same iteration and Gauss-Jordan elimination as k_rh, with the matrix held as float
// pairs (hi + lo, ~48-bit significand) and all arithmetic on the float pipes: on GB300 a
// warp-wide FP64 instruction issues at ~1/64 of the float rate, and the elimination is
// pure multiply-add. Products are formed exactly (p = a*b, e = fma(a, b, -p), cross terms
// folded into e) and each output is renormalised once; the pivot reciprocal takes one
// Newton step r = x + x (1 - d x) from the float reciprocal x, which doubles its 24
// correct bits. Pivots are chosen on the high words.
struct cdf {
  df64 re, im;
};

__device__ __forceinline__ df64 df_recip(df64 d) {
  const float x = __frcp_rn(d.hi);
  const df64 e = df64{1.f, 0.f} - d * x;
  return df64{x, 0.f} + e * x;
}

__device__ __forceinline__ cdf e_load(const float4* p) {
  const float4 v = *p;
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ df64 e_load(const float2* p) {
  const float2 v = *p;
  return {v.x, v.y};
}
__device__ __forceinline__ void e_store(float4* p, cdf a) { *p = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__device__ __forceinline__ void e_store(float2* p, df64 a) { *p = make_float2(a.hi, a.lo); }
__device__ __forceinline__ float e_abs2hi(cdf a) { return a.re.hi * a.re.hi + a.im.hi * a.im.hi; }
__device__ __forceinline__ float e_abs2hi(df64 a) { return a.hi * a.hi; }
__device__ __forceinline__ cdf e_zero(cdf) { return {df_zero(), df_zero()}; }
__device__ __forceinline__ df64 e_zero(df64) { return df_zero(); }
// w - f r
__device__ __forceinline__ cdf e_submul(cdf w, cdf f, cdf r) {
  return {df_axpy2(w.re, -f.re, r.re, f.im, r.im), df_axpy2(w.im, -f.re, r.im, -f.im, r.re)};
}
__device__ __forceinline__ df64 e_submul(df64 w, df64 f, df64 r) { return df_axpy1(w, -f, r); }
__device__ __forceinline__ cdf e_mul(cdf a, cdf b) {
  return {df_axpy2(df_zero(), a.re, b.re, -a.im, b.im), df_axpy2(df_zero(), a.re, b.im, a.im, b.re)};
}
__device__ __forceinline__ df64 e_mul(df64 a, df64 b) { return a * b; }
__device__ __forceinline__ cdf e_inv(cdf a) {
  const df64 r = df_recip(df_axpy2(df_zero(), a.re, a.re, a.im, a.im));
  return {a.re * r, -(a.im * r)};
}
__device__ __forceinline__ df64 e_inv(df64 a) { return df_recip(a); }
// (a + b) / 2 and |(a + b) / 2 - a|^2, |(a + b) / 2|^2 (high words)
__device__ __forceinline__ cdf e_avg(cdf a, cdf b, float& d2, float& n2) {
  const cdf s = {df_half(a.re + b.re), df_half(a.im + b.im)};
  const float dr = __fsub_rn(s.re.hi, a.re.hi), di = __fsub_rn(s.im.hi, a.im.hi);
  d2 += dr * dr + di * di;
  n2 += e_abs2hi(s);
  return s;
}
__device__ __forceinline__ df64 e_avg(df64 a, df64 b, float& d2, float& n2) {
  const df64 s = df_half(a + b);
  const float d = __fsub_rn(s.hi, a.hi);
  d2 += d * d;
  n2 += s.hi * s.hi;
  return s;
}
__device__ __forceinline__ cdf e_scale(cdf a, float f) { return {a.re * f, a.im * f}; }
__device__ __forceinline__ df64 e_scale(df64 a, float f) { return a * f; }
// (g a + b / g) / 2 with |(...) - a|^2 and |(...)|^2 (high words), g > 0
__device__ __forceinline__ cdf e_avg_scaled(cdf a, cdf b, float g, float gi, float& d2, float& n2) {
  const cdf sa = e_scale(a, g), sb = e_scale(b, gi);
  const cdf s = {df_half(sa.re + sb.re), df_half(sa.im + sb.im)};
  const float dr = __fsub_rn(s.re.hi, a.re.hi), di = __fsub_rn(s.im.hi, a.im.hi);
  d2 += dr * dr + di * di;
  n2 += e_abs2hi(s);
  return s;
}
__device__ __forceinline__ df64 e_avg_scaled(df64 a, df64 b, float g, float gi, float& d2, float& n2) {
  const df64 s = df_half(e_scale(a, g) + e_scale(b, gi));
  const float d = __fsub_rn(s.hi, a.hi);
  d2 += d * d;
  n2 += s.hi * s.hi;
  return s;
}
__device__ __forceinline__ bool e_finite(cdf a) {
  return isfinite(a.re.hi) && isfinite(a.re.lo) && isfinite(a.im.hi) && isfinite(a.im.lo);
}
__device__ __forceinline__ bool e_finite(df64 a) { return isfinite(a.hi) && isfinite(a.lo); }
__device__ __forceinline__ double2 e_to2(cdf a) { return make_double2(df_to_double(a.re), df_to_double(a.im)); }
__device__ __forceinline__ double2 e_to2(df64 a) { return make_double2(df_to_double(a), 0.0); }
__device__ __forceinline__ cdf e_from2(double2 v, cdf) { return {df_from_double(v.x), df_from_double(v.y)}; }
__device__ __forceinline__ df64 e_from2(double2 v, df64) { return df_from_double(v.x); }

template <bool CPLX>
struct RhDf;
template <> struct RhDf<true> { using E = cdf; using St = float4; };
template <> struct RhDf<false> { using E = df64; using St = float2; };

template <bool CPLX>
__global__ void __launch_bounds__(1024) k_rh_df(int count, int dense_m, const double2* __restrict__ dense_T,
                                                InnerWork w, int dl, double rh_tol, int rh_maxit, int mid0,
                                                int scale) {
  using E = typename RhDf<CPLX>::E;
  using St = typename RhDf<CPLX>::St;
  extern __shared__ __align__(16) unsigned char smem[];
  const int mid = mid0 + blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  int m;
  if (dense_m > 0) {
    m = dense_m;
  } else {
    const int prob = mid % count;
    const int le = w.leff[prob];
    m = mid < count ? le : le - dl;
  }
  if (m <= 0) {
    if (tid == 0) { w.rh_ok[mid] = m == 0 ? 0 : 1; w.rh_its[mid] = 0; }
    return;
  }
  St* W = (St*)smem;                  // m x m working matrix
  St* col = W + (size_t)m * m;        // column buffer / reduction scratch
  double* red = (double*)col;
  __shared__ int s_piv;
  __shared__ St s_inv, s_djj;
  __shared__ float s_logdet;  // log |det S_n| from the pivots (high words)
  // global S_n (row-major, leading dim m) in the float-pair storage, in the problem's
  // double2 slot (16 bytes per element)
  St* Sg = (St*)(w.S + (size_t)mid * kMaxL * kMaxL);
  int* perm = w.perm + (size_t)mid * kMaxL;
  const E ez = e_zero(E{});
  for (int e = tid; e < m * m; e += nth) {
    const int i = e / m, j = e % m;
    double2 v = make_double2(0.0, 0.0);
    if (dense_m > 0) {
      v = dense_T[(size_t)mid * m * m + e];
    } else {
      const double2* T = w.T + (size_t)(mid % count) * kMaxL * 3;
      if (i == j) v = T[i * 3 + 0];
      else if (i == j + 1) v = T[i * 3 + 1];
      else if (j == i + 1) v = T[j * 3 + 2];
    }
    e_store(&Sg[e], e_from2(v, ez));
  }
  __syncthreads();
  int ok = 0, it = 0;
  float rel_prev = INFINITY;  // ||S_n - S_{n-1}|| / ||S_n|| of the last iteration
  // the elimination's element share of thread tid >= 32 (warps 1..): the elements
  // u, u + nth - 32, ... of the (m - 1) x (m - 1) block, row-major (u = tid - 32)
  const int mm = m - 1;
  const int fu = tid - 32, fst = nth - 32;
  const int fr0 = (mm > 0 && fu >= 0) ? fu / mm : 0, fc0 = (mm > 0 && fu >= 0) ? fu % mm : 0;
  const int fdr = mm > 0 ? fst / mm : 0, fdc = mm > 0 ? fst % mm : 0;
  for (it = 1; it <= rh_maxit; ++it) {
    for (int e = tid; e < m * m; e += nth) W[e] = Sg[e];
    __syncthreads();
    bool singular = false;
    // Gauss-Jordan with partial pivoting, two barriers a column: (A) the pivot row is
    // swapped into row j and scaled, the multipliers of column j saved; (B) every other row
    // is eliminated, while warp 0 eliminates column j + 1 and chooses its pivot (its row
    // p, 1 / W[p][j+1] and the old diagonal W[j+1][j+1] go through s_piv, s_inv, s_djj).
    auto pivot_of = [&](int jc, int lane, float best, int bi) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      __syncwarp();
      if (lane == 0) {
        s_piv = best > 0.f ? bi : -1;
        if (best > 0.f) {
          s_inv = W[(size_t)bi * m + jc];
          s_djj = W[(size_t)jc * m + jc];
          s_logdet = (jc == 0 ? 0.f : s_logdet) + 0.5f * __logf(best);
        }
      }
    };
    if (tid < 32) {
      float best = -1.f;
      int bi = 0;
      for (int i = tid; i < m; i += 32) {
        const float a2 = e_abs2hi(e_load(&W[(size_t)i * m]));
        if (a2 > best) { best = a2; bi = i; }
      }
      pivot_of(0, tid, best, bi);
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
      const int p = s_piv;
      if (p < 0) { singular = true; break; }
      const E inv = e_inv(e_load(&s_inv));
      const St djj = s_djj;
      if (tid == 0) perm[j] = p;
      // (A) rows j and p are touched column by column by one thread each; the multipliers
      // read column j of the other rows (row p's multiplier is the old W[j][j])
      for (int c = tid; c < m; c += nth) {
        const E wp = e_load(&W[(size_t)p * m + c]);
        const St wj = W[(size_t)j * m + c];
        e_store(&W[(size_t)j * m + c], c == j ? inv : e_mul(wp, inv));
        if (p != j) W[(size_t)p * m + c] = wj;
      }
      for (int i = tid; i < m; i += nth) col[i] = i == j ? St{} : (i == p ? djj : W[(size_t)i * m + j]);
      __syncthreads();
      // (B) W[i][c] -= col[i] W[j][c] for i != j; column j becomes -col[i] / pivot (the
      // inverse's column, in place). Warp 0 takes column cw = j + 1 (j itself at the last
      // column) and, for j + 1 < m, picks that column's pivot; warps 1.. share the other
      // (m - 1) x (m - 1) elements evenly (rows without j, columns without cw).
      {
        const int tx = tid & 31;
        const int cw = j + 1 < m ? j + 1 : j;
        if (tid >= 32) {
          if (mm > 0) {
            int ri = fr0, ci = fc0;
            while (ri < mm) {
              const int i = ri + (ri >= j);
              const int c = ci + (ci >= cw);
              const E f = e_load(&col[i]);
              const E pj = e_load(&W[(size_t)j * m + c]);
              e_store(&W[(size_t)i * m + c], e_submul(c == j ? ez : e_load(&W[(size_t)i * m + c]), f, pj));
              ri += fdr;
              ci += fdc;
              if (ci >= mm) {
                ci -= mm;
                ++ri;
              }
            }
          }
        } else {
          const E pj1 = e_load(&W[(size_t)j * m + cw]);
          float best = -1.f;
          int bi = j + 1;
          for (int i = tx; i < m; i += 32) {
            if (i == j) continue;
            const E v = e_submul(cw == j ? ez : e_load(&W[(size_t)i * m + cw]), e_load(&col[i]), pj1);
            e_store(&W[(size_t)i * m + cw], v);
            if (cw == j + 1 && i > j) {
              const float a2 = e_abs2hi(v);
              if (a2 > best) { best = a2; bi = i; }
            }
          }
          if (cw == j + 1) pivot_of(j + 1, tx, best, bi);
        }
      }
      __syncthreads();
    }
    if (singular) { ok = 0; break; }
    // the row interchanges permute the inverse's columns: undo them all in one gather,
    // idx[c] = the column that ends at c (the interchanges applied in reverse order)
    int* idx = (int*)col;
    if (tid == 0) {
      for (int c = 0; c < m; ++c) idx[c] = c;
      for (int j = m - 1; j >= 0; --j) {
        const int pj = perm[j];
        const int t = idx[j];
        idx[j] = idx[pj];
        idx[pj] = t;
      }
    }
    __syncthreads();
    {
      const int tx = tid & 31, ty = tid >> 5;
      for (int i = ty; i < m; i += 32) {
        St v[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int c = tx + 32 * b;
          if (c < m) v[b] = W[(size_t)i * m + idx[c]];
        }
        __syncwarp();
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int c = tx + 32 * b;
          if (c < m) W[(size_t)i * m + c] = v[b];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    float d2 = 0.f, n2 = 0.f;
    bool fin = true;
    // determinant scaling (Byers; Kenney and Laub, SIAM J. Matrix Anal. Appl. 13 (1992)):
    // S_{n+1} = (g S_n + S_n^{-1} / g) / 2 with g = |det S_n|^{-1/m} while the iterate still
    // changes by more than 1e-2, the plain step of Eq. (Roberts) after that (its quadratic
    // convergence is untouched). The limit is sgn(S_0) either way.
    const float g = (scale && rel_prev > 1e-2f) ? __expf(-s_logdet / (float)m) : 1.f;
    const float gi = 1.f / g;
    for (int e = tid; e < m * m; e += nth) {
      const E a = e_load(&Sg[e]);
      const E s1 = g == 1.f ? e_avg(a, e_load(&W[e]), d2, n2) : e_avg_scaled(a, e_load(&W[e]), g, gi, d2, n2);
      fin = fin && e_finite(s1);
      e_store(&Sg[e], s1);
    }
    __syncthreads();
    double dif = warp_sum((double)d2);
    double nrm = warp_sum((double)n2);
    const int fin_all = __syncthreads_and(fin ? 1 : 0);
    if ((tid & 31) == 0) { red[(tid >> 5) * 2] = dif; red[(tid >> 5) * 2 + 1] = nrm; }
    __syncthreads();
    double D = 0.0, N = 0.0;
    for (int q = 0; q < (nth >> 5); ++q) { D += red[2 * q]; N += red[2 * q + 1]; }
    __syncthreads();
    if (!fin_all || !isfinite(D) || !isfinite(N)) { ok = 0; break; }
    if (sqrt(D) <= rh_tol * sqrt(N)) { ok = 1; break; }
    rel_prev = (float)(sqrt(D) / sqrt(N));
  }
  if (tid == 0) {
    w.rh_ok[mid] = ok;
    w.rh_its[mid] = it > rh_maxit ? rh_maxit : it;
  }
  for (int i = tid; i < m; i += nth) w.s[(size_t)mid * kMaxL + i] = e_to2(e_load(&Sg[(size_t)i * m]));
  if (CPLX && dense_m > 0) {
    // the caller reads S as double2: convert in place (same 16-byte slot per element)
    __syncthreads();
    double2* Sd = w.S + (size_t)mid * kMaxL * kMaxL;
    for (int e = tid; e < m * m; e += nth) {
      const E v = e_load(&Sg[e]);
      Sd[e] = e_to2(v);
    }
  }
}

// ------------------------------------------------- inner Krylov in double-float
// k_inner with every operation on the float pipes: the tridiagonal factorisation and the
// two serial solves per step (the critical path of the inner level) and the vector
// updates in float pairs, the block reductions in float pairs. Square roots take one
// Newton step y + (x - y^2) / (2 y) from the float root, quotients multiply by the
// refined reciprocal (Karp and Markstein, ACM TOMS 23 (1997)). Outputs (T, Q) are double.
__device__ __forceinline__ cdf c_add(cdf a, cdf b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cdf c_conj(cdf a) { return {a.re, -a.im}; }
__device__ __forceinline__ cdf c_scale(cdf a, df64 s) { return {a.re * s, a.im * s}; }
// a + f r
__device__ __forceinline__ cdf c_addmul(cdf a, cdf f, cdf r) {
  return {df_axpy2(a.re, f.re, r.re, -f.im, r.im), df_axpy2(a.im, f.re, r.im, f.im, r.re)};
}
// a + conj(f) r
__device__ __forceinline__ cdf c_addmulc(cdf a, cdf f, cdf r) {
  return {df_axpy2(a.re, f.re, r.re, f.im, r.im), df_axpy2(a.im, f.re, r.im, -f.im, r.re)};
}
// a - conj(f) r
__device__ __forceinline__ cdf c_submulc(cdf a, cdf f, cdf r) {
  return {df_axpy2(a.re, -f.re, r.re, -f.im, r.im), df_axpy2(a.im, -f.re, r.im, f.im, r.re)};
}
__device__ __forceinline__ df64 df_sqrt(df64 x) {
  if (!(x.hi > 0.f)) return df_zero();
  const float y = __fsqrt_rn(x.hi);
  const df64 e = x - df_prod(y, y);
  return df_two_sum(y, __fmul_rn(e.hi, __fdiv_rn(0.5f, y)));
}
__device__ __forceinline__ df64 block_sum_df(df64 v, df64* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  df64 s = df_zero();
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = s + red[w];
  return s;
}

struct InnerSmemDf {
  float4 *d, *a, *c, *uinv, *u1, *u2, *l, *q, *qp, *w, *wp, *u, *z;
  unsigned char* sw;
  df64* red;
};

__device__ bool tri_factor_df(const InnerSmemDf& S, int k) {
  const cdf zero = {df_zero(), df_zero()};
  cdf dd = e_load(&S.d[0]);
  cdf ee = k > 1 ? e_load(&S.c[0]) : zero;
  for (int m = 0; m < k - 1; ++m) {
    const cdf an = e_load(&S.a[m + 1]), dn = e_load(&S.d[m + 1]);
    const cdf cn = (m + 1 <= k - 2) ? e_load(&S.c[m + 1]) : zero;
    cdf r0, r1, r2, lm;
    if (e_abs2hi(dd) >= e_abs2hi(an)) {
      if (e_abs2hi(dd) == 0.f) return false;
      lm = e_mul(an, e_inv(dd));
      r0 = dd; r1 = ee; r2 = zero;
      dd = e_submul(dn, lm, ee);
      ee = cn;
      S.sw[m] = 0;
    } else {
      lm = e_mul(dd, e_inv(an));
      r0 = an; r1 = dn; r2 = cn;
      dd = e_submul(ee, lm, dn);
      ee = e_submul(zero, lm, cn);
      S.sw[m] = 1;
    }
    // U = D (1 + N) with D = diag(r0): the solves need 1 / r0 and the rows of N, r1 / r0
    // and r2 / r0, so that each step of their serial recurrences is one multiply-add
    const cdf ri = e_inv(r0);
    e_store(&S.uinv[m], ri);
    e_store(&S.u1[m], e_mul(r1, ri));
    e_store(&S.u2[m], e_mul(r2, ri));
    e_store(&S.l[m], lm);
  }
  if (e_abs2hi(dd) == 0.f) return false;
  e_store(&S.uinv[k - 1], e_inv(dd));
  return true;
}

// x = H^{-1} b in three parts: the row interchanges and L (serial, one thread), the scaling
// by 1 / diag(U) (all threads), then (1 + N) x = g backwards (serial). Each serial step is
// one complex multiply-add on the recurrence's critical path.
__device__ void tri_solve_fwd_df(const InnerSmemDf& S, int k, const float4* b, float4* x) {
  cdf cur = e_load(&b[0]);
#pragma unroll 2
  for (int m = 0; m < k - 1; ++m) {
    const cdf nb = e_load(&b[m + 1]);
    const bool sw = S.sw[m];
    const cdf bsel = sw ? nb : cur, asel = sw ? cur : nb;
    e_store(&x[m], bsel);
    cur = e_submul(asel, e_load(&S.l[m]), bsel);
  }
  e_store(&x[k - 1], cur);
}
__device__ void tri_solve_bwd_df(const InnerSmemDf& S, int k, float4* x) {
  if (k < 2) return;
  cdf x1 = e_load(&x[k - 1]);
  cdf x0 = e_submul(e_load(&x[k - 2]), e_load(&S.u1[k - 2]), x1);
  e_store(&x[k - 2], x0);
#pragma unroll 2
  for (int m = k - 3; m >= 0; --m) {
    const cdf xm = e_submul(e_submul(e_load(&x[m]), e_load(&S.u2[m]), x1), e_load(&S.u1[m]), x0);
    e_store(&x[m], xm);
    x1 = x0;
    x0 = xm;
  }
}

// z = H^{-dag} b: U^dag = (1 + N)^dag D^dag, so (1 + N^dag) y = b forwards (serial), z =
// conj(1 / diag(U)) y (all threads), then the interchanges' adjoints backwards (serial)
__device__ void tri_solve_dag_fwd_df(const InnerSmemDf& S, int k, const float4* b, float4* z) {
  const cdf zero = {df_zero(), df_zero()};
  cdf z1 = zero, z2 = zero;  // y[m-1], y[m-2]
#pragma unroll 2
  for (int m = 0; m < k; ++m) {
    cdf t = e_load(&b[m]);
    if (m >= 2) t = c_submulc(t, e_load(&S.u2[m - 2]), z2);
    if (m >= 1) t = c_submulc(t, e_load(&S.u1[m - 1]), z1);
    e_store(&z[m], t);
    z2 = z1;
    z1 = t;
  }
}
__device__ void tri_solve_dag_bwd_df(const InnerSmemDf& S, int k, float4* z) {
  cdf gn = e_load(&z[k - 1]);  // current z[m + 1]
#pragma unroll 2
  for (int m = k - 2; m >= 0; --m) {
    const cdf v = c_submulc(e_load(&z[m]), e_load(&S.l[m]), gn);
    const bool sw = S.sw[m];
    e_store(&z[m + 1], sw ? v : gn);
    gn = sw ? gn : v;
  }
  e_store(&z[0], gn);
}

__global__ void __launch_bounds__(kInnerThreads) k_inner_df(const int* __restrict__ k_dev,
                                                            const int* __restrict__ l_dev, int hermitian,
                                                            const double2* __restrict__ alp,
                                                            const double2* __restrict__ bet,
                                                            const double2* __restrict__ gam, int ldc, InnerWork w) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int prob = blockIdx.x;
  const int k = k_dev[prob];
  const int l = min(l_dev[prob], k);
  const int tid = threadIdx.x;
  InnerSmemDf S;
  {
    float4* base = (float4*)smem;
    S.d = base; S.a = base + k; S.c = base + 2 * k;
    S.uinv = base + 3 * k; S.u1 = base + 4 * k; S.u2 = base + 5 * k; S.l = base + 6 * k;
    S.q = base + 7 * k; S.qp = base + 8 * k; S.w = base + 9 * k; S.wp = base + 10 * k;
    S.u = base + 11 * k; S.z = base + 12 * k;
    S.red = (df64*)(base + 13 * k);
    S.sw = (unsigned char*)(S.red + 32);
  }
  const cdf zero = {df_zero(), df_zero()};
  const double2* al = alp + (size_t)prob * ldc;
  const double2* be = bet + (size_t)prob * ldc;
  const double2* ga = gam + (size_t)prob * ldc;
  for (int m = tid; m < k; m += blockDim.x) {
    double2 dm = al[m + 1];
    double2 am = m >= 1 ? be[m + 1] : make_double2(0.0, 0.0);
    double2 cm = m + 1 < k ? ga[m + 2] : make_double2(0.0, 0.0);
    if (hermitian) { dm.y = 0.0; am.y = 0.0; cm = m + 1 < k ? make_double2(be[m + 2].x, 0.0) : cm; }
    e_store(&S.d[m], e_from2(dm, zero));
    e_store(&S.a[m], e_from2(am, zero));
    e_store(&S.c[m], e_from2(cm, zero));
    const cdf q0 = m == 0 ? cdf{{1.f, 0.f}, df_zero()} : zero;
    e_store(&S.q[m], q0);
    e_store(&S.w[m], q0);
    e_store(&S.qp[m], zero);
    e_store(&S.wp[m], zero);
  }
  __syncthreads();
  __shared__ int s_ok;
  if (tid == 0) s_ok = tri_factor_df(S, k) ? 1 : 0;
  __syncthreads();
  if (!s_ok) {
    if (tid == 0) { w.fail[prob] = 1; w.leff[prob] = 0; }
    return;
  }
  double2* Q = w.Q + (size_t)prob * w.ld * kMaxL;
  double2* T = w.T + (size_t)prob * kMaxL * 3;
  df64 b_i = df_zero();
  cdf g_i = zero;
  int done = 0;
  const float exhaust_tol = 1e-13f;
  for (int i = 0; i < l; ++i) {
    for (int m = tid; m < k; m += blockDim.x) Q[(size_t)m * kMaxL + i] = e_to2(e_load(&S.q[m]));
    if (tid == 0) tri_solve_fwd_df(S, k, S.q, S.u);
    if (!hermitian && tid == 32) tri_solve_dag_fwd_df(S, k, S.w, S.z);
    __syncthreads();
    for (int m = tid; m < k; m += blockDim.x) {
      const cdf ri = e_load(&S.uinv[m]);
      e_store(&S.u[m], e_mul(e_load(&S.u[m]), ri));
      if (!hermitian) e_store(&S.z[m], e_mul(e_load(&S.z[m]), c_conj(ri)));
    }
    __syncthreads();
    if (tid == 0) tri_solve_bwd_df(S, k, S.u);
    if (!hermitian && tid == 32) tri_solve_dag_bwd_df(S, k, S.z);
    __syncthreads();
    float mq2 = 0.f;
    for (int m = tid; m < k; m += blockDim.x) {
      cdf t = e_mul(e_load(&S.d[m]), e_load(&S.q[m]));
      if (m >= 1) t = c_addmul(t, e_load(&S.a[m]), e_load(&S.q[m - 1]));
      if (m + 1 < k) t = c_addmul(t, e_load(&S.c[m]), e_load(&S.q[m + 1]));
      t = c_add(t, e_load(&S.u[m]));
      mq2 += e_abs2hi(t);
      const cdf qp = e_load(&S.qp[m]);
      e_store(&S.u[m], hermitian ? e_submul(t, cdf{b_i, df_zero()}, qp) : e_submul(t, g_i, qp));  // p
      if (!hermitian) {
        cdf y = e_mul(c_conj(e_load(&S.d[m])), e_load(&S.w[m]));
        if (m >= 1) y = c_addmulc(y, e_load(&S.c[m - 1]), e_load(&S.w[m - 1]));
        if (m + 1 < k) y = c_addmulc(y, e_load(&S.a[m + 1]), e_load(&S.w[m + 1]));
        y = c_add(y, e_load(&S.z[m]));
        e_store(&S.z[m], e_submul(y, cdf{b_i, df_zero()}, e_load(&S.wp[m])));  // r
      }
    }
    __syncthreads();
    // alpha = w^dag p (q^dag p in the Hermitian case)
    df64 are = df_zero(), aim = df_zero();
    for (int m = tid; m < k; m += blockDim.x) {
      const cdf wm = e_load(hermitian ? &S.q[m] : &S.w[m]);
      const cdf pm = e_load(&S.u[m]);
      are = df_axpy2(are, wm.re, pm.re, wm.im, pm.im);
      aim = df_axpy2(aim, wm.re, pm.im, -wm.im, pm.re);
    }
    are = block_sum_df(are, S.red);
    aim = hermitian ? df_zero() : block_sum_df(aim, S.red);
    const df64 mqn = df_sqrt(block_sum_df(df64{mq2, 0.f}, S.red));
    const cdf a_i = {are, aim};
    if (tid == 0) T[i * 3 + 0] = e_to2(a_i);
    done = i + 1;
    if (i == l - 1) break;
    // q~ = p - alpha q ; w~ = r - conj(alpha) w ; delta = w~^dag q~
    df64 dre = df_zero(), dim = df_zero(), n2 = df_zero();
    for (int m = tid; m < k; m += blockDim.x) {
      const cdf qt = e_submul(e_load(&S.u[m]), a_i, e_load(&S.q[m]));
      e_store(&S.u[m], qt);
      if (hermitian) {
        n2 = df_axpy2(n2, qt.re, qt.re, qt.im, qt.im);
      } else {
        const cdf wt = c_submulc(e_load(&S.z[m]), a_i, e_load(&S.w[m]));
        e_store(&S.z[m], wt);
        dre = df_axpy2(dre, wt.re, qt.re, wt.im, qt.im);
        dim = df_axpy2(dim, wt.re, qt.im, -wt.im, qt.re);
      }
    }
    df64 bn;
    cdf gn;
    if (hermitian) {
      bn = df_sqrt(block_sum_df(n2, S.red));
      gn = {bn, df_zero()};
    } else {
      dre = block_sum_df(dre, S.red);
      dim = block_sum_df(dim, S.red);
      bn = df_sqrt(df_sqrt(df_axpy2(df_zero(), dre, dre, dim, dim)));
      const df64 rb = bn.hi > 0.f ? df_recip(bn) : df_zero();
      gn = {dre * rb, dim * rb};
    }
    if (!(bn.hi > exhaust_tol * mqn.hi)) break;  // inner space exhausted: T_i is exact
    if (tid == 0) {
      T[(i + 1) * 3 + 1] = make_double2(df_to_double(bn), 0.0);
      T[(i + 1) * 3 + 2] = e_to2(gn);
    }
    const cdf wdiv = e_inv(c_conj(gn));
    const df64 rbn = df_recip(bn);
    __syncthreads();
    for (int m = tid; m < k; m += blockDim.x) {
      e_store(&S.qp[m], e_load(&S.q[m]));
      e_store(&S.q[m], c_scale(e_load(&S.u[m]), rbn));
      if (!hermitian) {
        e_store(&S.wp[m], e_load(&S.w[m]));
        e_store(&S.w[m], e_mul(e_load(&S.z[m]), wdiv));
      }
    }
    b_i = bn;
    g_i = gn;
    __syncthreads();
  }
  if (tid == 0) {
    w.leff[prob] = done;
    T[0 * 3 + 1] = make_double2(0.0, 0.0);
    T[0 * 3 + 2] = make_double2(0.0, 0.0);
    w.fail[prob] = 0;
  }
}

// ------------------------------------------------------------ combine
__global__ void __launch_bounds__(kInnerThreads) k_combine(int count, const int* __restrict__ k_dev,
                                                           const int* __restrict__ l_dev, InnerWork w, int dl,
                                                           double2* c, int ldo, void* cacc, const double* nv,
                                                           int ldn, int prec,
                                                           double* est_inner, const double2* cprev, int ldp,
                                                           const int* kprev_dev, double* est_outer, int* rh_status,
                                                           int* rh_iters, int have_est) {
  const int* fail = w.fail;
  __shared__ double red[32];
  const int prob = blockIdx.x;
  const int k = k_dev[prob];
  const int le = w.leff[prob];
  const int le2 = le - dl;
  const int tid = threadIdx.x;
  const double2* Q = w.Q + (size_t)prob * w.ld * kMaxL;
  const double2* s1 = w.s + (size_t)prob * kMaxL;
  const double2* s2 = w.s + (size_t)(count + prob) * kMaxL;
  const bool bad = fail[prob] != 0 || le <= 0 || !w.rh_ok[prob];
  // the inner space is exact when it was exhausted early or spans all of C^k
  const bool exact = le >= k || le < min(l_dev[prob], k);
  double nc = 0.0, nd = 0.0, no = 0.0;
  const int kp = kprev_dev ? kprev_dev[prob] : 0;
  // entries k+1 .. ldo-1 are cleared so that a shorter c never carries stale values
  for (int m = k + tid; m < ldo - 1; m += blockDim.x) {
    c[(size_t)prob * ldo + m + 1] = make_double2(0.0, 0.0);
    if (cacc) {
      if (prec == OV_PREC_FP64) ((double2*)cacc)[(size_t)prob * ldo + m + 1] = make_double2(0.0, 0.0);
      else ((float4*)cacc)[(size_t)prob * ldo + m + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  for (int m = tid; m < k; m += blockDim.x) {
    double2 v = make_double2(0.0, 0.0), v2 = make_double2(0.0, 0.0);
    if (!bad) {
      for (int i = 0; i < le; ++i) {
        const double2 qv = Q[(size_t)m * kMaxL + i];
        v = zadd(v, zmul(qv, s1[i]));
        if (have_est && i < le2) v2 = zadd(v2, zmul(qv, s2[i]));
      }
    }
    c[(size_t)prob * ldo + m + 1] = v;
    if (cacc) {
      // the recombination sums c_j v_j = (c_j / nv_j) t_j over the unnormalised basis
      const double sc = nv ? 1.0 / nv[(size_t)prob * ldn + m + 1] : 1.0;
      const double2 vs = make_double2(v.x * sc, v.y * sc);
      if (prec == OV_PREC_FP64) {
        ((double2*)cacc)[(size_t)prob * ldo + m + 1] = vs;
      } else {
        const df64 re = df_from_double(vs.x), im = df_from_double(vs.y);
        ((float4*)cacc)[(size_t)prob * ldo + m + 1] = make_float4(re.hi, re.lo, im.hi, im.lo);
      }
    }
    nc += zabs2(v);
    if (le2 >= 1) nd += zabs2(zsub(v, v2));
    if (kp > 0 && cprev) {
      const double2 pv = m < kp ? cprev[(size_t)prob * ldp + m + 1] : make_double2(0.0, 0.0);
      no += zabs2(zsub(v, pv));
    }
  }
  nc = block_sum(nc, red);
  nd = block_sum(nd, red);
  no = block_sum(no, red);
  if (tid == 0) {
    const double cn = sqrt(nc);
    // inner estimate: 0 when the inner space is exact (exhausted or l_eff = k)
    double ei;
    if (bad) ei = INFINITY;
    else if (exact) ei = 0.0;
    else if (!have_est) ei = NAN;
    else if (le2 < 1 || w.rh_ok[count + prob] == 0) ei = INFINITY;
    else ei = sqrt(nd) / cn;
    est_inner[prob] = ei;
    if (est_outer) est_outer[prob] = (kp > 0 && cprev && !bad) ? sqrt(no) / cn : INFINITY;
    rh_status[prob] = bad ? (fail[prob] ? 2 : 1) : 0;
    rh_iters[prob] = w.rh_its[prob];
  }
}

static size_t inner_smem(int k) { return (size_t)13 * k * sizeof(double2) + 32 * sizeof(double) + k + 16; }

cudaError_t run_inner(int count, const int* k_dev, const int* l_dev, int hermitian, const double2* alp,
                      const double2* bet, const double2* gam, const double* nv, int ldc, InnerWork& w,
                      double rh_tol, int rh_maxit, int inner_dl, double2* c, int ldo, void* cacc, int prec,
                      double* est_inner,
                      const double2* cprev, int ldp, const int* kprev_dev, double* est_outer, int* rh_status,
                      int* rh_iters, int phase, cudaStream_t st) {
  cudaError_t e;
  if (phase != 2) {
    const size_t sm = inner_smem(w.ld);  // float pairs take the bytes of the doubles they replace
    if (w.arith == OV_INNER_DF64) {
      e = cudaFuncSetAttribute(k_inner_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      k_inner_df<<<count, kInnerThreads, sm, st>>>(k_dev, l_dev, hermitian, alp, bet, gam, ldc, w);
    } else {
      e = cudaFuncSetAttribute(k_inner, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      k_inner<<<count, kInnerThreads, sm, st>>>(k_dev, l_dev, hermitian, alp, bet, gam, ldc, w);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // phase 0: both Roberts-Higham sets (the matrices and their leading l - dl blocks);
  // phase 1: the matrices only (no inner estimate); phase 2: only the leading blocks
  // of the matrices left by a phase-1 call (the inner estimate on request)
  const int mid0 = phase == 2 ? count : 0;
  const int nmat = phase == 0 ? 2 * count : count;
  const size_t esz = hermitian ? sizeof(double) : sizeof(double2);
  // matrix + column buffer (which also holds the 64-double reduction scratch)
  const size_t rsm = (size_t)kMaxL * kMaxL * esz + std::max<size_t>(kMaxL * esz, 512);
  if (w.arith == OV_INNER_DF64) {
    // float pairs take the bytes of the double elements they replace
    if (hermitian) {
      e = cudaFuncSetAttribute(k_rh_df<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
      if (e != cudaSuccess) return e;
      k_rh_df<false><<<nmat, 1024, rsm, st>>>(count, 0, nullptr, w, inner_dl, rh_tol, rh_maxit, mid0, w.rh_scale);
    } else {
      e = cudaFuncSetAttribute(k_rh_df<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
      if (e != cudaSuccess) return e;
      k_rh_df<true><<<nmat, 1024, rsm, st>>>(count, 0, nullptr, w, inner_dl, rh_tol, rh_maxit, mid0, w.rh_scale);
    }
  } else if (hermitian) {
    e = cudaFuncSetAttribute(k_rh<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
    if (e != cudaSuccess) return e;
    k_rh<false><<<nmat, 1024, rsm, st>>>(count, 0, nullptr, w, inner_dl, rh_tol, rh_maxit, mid0);
  } else {
    e = cudaFuncSetAttribute(k_rh<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
    if (e != cudaSuccess) return e;
    k_rh<true><<<nmat, 1024, rsm, st>>>(count, 0, nullptr, w, inner_dl, rh_tol, rh_maxit, mid0);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_combine<<<count, kInnerThreads, 0, st>>>(count, k_dev, l_dev, w, inner_dl, c, ldo, cacc, nv, ldc, prec, est_inner,
                                             cprev, ldp, kprev_dev, est_outer, rh_status, rh_iters, phase != 1);
  return cudaGetLastError();
}

cudaError_t run_rh_dense(int count, int m, const double2* T, double2* S, int* iters, int* ok, double rh_tol,
                         int rh_maxit, InnerWork& w, cudaStream_t st) {
  const size_t rsm = (size_t)m * m * sizeof(double2) + std::max<size_t>(m * sizeof(double2), 512);
  cudaError_t e;
  if (w.arith == OV_INNER_DF64) {
    e = cudaFuncSetAttribute(k_rh_df<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
    if (e != cudaSuccess) return e;
    k_rh_df<true><<<count, 1024, rsm, st>>>(count, m, T, w, 0, rh_tol, rh_maxit, 0, 0);
  } else {
    e = cudaFuncSetAttribute(k_rh<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
    if (e != cudaSuccess) return e;
    k_rh<true><<<count, 1024, rsm, st>>>(count, m, T, w, 0, rh_tol, rh_maxit, 0);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int i = 0; i < count; ++i) {
    e = cudaMemcpy2DAsync(S + (size_t)i * m * m, sizeof(double2) * m * m, w.S + (size_t)i * kMaxL * kMaxL,
                          sizeof(double2) * m * m, sizeof(double2) * m * m, 1, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemcpyAsync(iters, w.rh_its, sizeof(int) * count, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(ok, w.rh_ok, sizeof(int) * count, cudaMemcpyDeviceToDevice, st);
}

}  // namespace ov
