// Outer Krylov level: the gamma5 Wilson-Dirac stencil fused with the Lanczos /
// two-sided Lanczos recurrences, vector updates with fixed-order reductions, and
// recombination of the result (Sec. 2, Eq. (approximation); Sec. 3, Eq. (nested)).
//
// Layout: an internal spinor field is [rhs][12][V] of the precision's storage type
// (component c = 3*spin + colour, site fastest), so a warp reads consecutive sites of
// one component (coalesced). Links are [4][9][V] (nu, a*3+b, site) with the
// antiperiodic t-boundary sign folded into U_t on the last time slice; the double-float
// mode keeps a second plane of low words 36 V elements further on.
//
// Precisions: FP64; FP32 (float vectors and links, double-float reductions); double-float
// (vectors and links as float pairs, compensated hop sums); and the relaxed double-float
// steps (the same storage and recurrence with the hop sum in float on the high words).
//
// Reductions: every block writes its partial sums (double) to a partials array; the
// last block of each right-hand side (atomic ticket, no spin-wait) adds the partials in
// a fixed order and writes the Krylov coefficient. Results are therefore bitwise
// reproducible run to run.
#include "ov_internal.h"
#include "ov_types.cuh"

namespace ov {

int num_site_blocks(const Geometry& g, int bs) { return (g.V + bs - 1) / bs; }

size_t vec_elem_bytes(int prec) {
  return prec == OV_PREC_FP32 ? sizeof(float2) : (prec == OV_PREC_FP64 ? sizeof(double2) : sizeof(float4));
}
size_t acc_elem_bytes(int prec) { return prec == OV_PREC_FP64 ? sizeof(double2) : sizeof(float4); }

template <class P> struct AccOf;
template <> struct AccOf<PrecF64> { using A = double; using st = double2; };
template <> struct AccOf<PrecF32> { using A = df64; using st = float4; };
template <> struct AccOf<PrecDF64> { using A = df64; using st = float4; };
template <> struct AccOf<PrecDF64R> { using A = df64; using st = float4; };

__device__ __forceinline__ cx<double> ld_acc(const double2* p) { double2 v = *p; return {v.x, v.y}; }
__device__ __forceinline__ cx<df64> ld_acc(const float4* p) { float4 v = *p; return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ void st_acc(double2* p, cx<double> a) { *p = make_double2(a.re, a.im); }
__device__ __forceinline__ void st_acc(float4* p, cx<df64> a) { *p = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }

// p - a v in one fused step per component (double-float: both products exact, one
// renormalisation)
template <class R> __device__ __forceinline__ cx<R> csubmul(cx<R> p, cx<R> a, cx<R> v) { return p - cmul(a, v); }
__device__ __forceinline__ cx<df64> csubmul(cx<df64> p, cx<df64> a, cx<df64> v) {
  return {df_axpy2(p.re, -a.re, v.re, a.im, v.im), df_axpy2(p.im, -a.re, v.im, -a.im, v.re)};
}
// acc += |t|^2
__device__ __forceinline__ void acc_norm(double& acc, cx<double> t) { acc = fma(t.re, t.re, fma(t.im, t.im, acc)); }
__device__ __forceinline__ void acc_norm(df64& acc, cx<float> t) { acc = df_axpy2(acc, t.re, t.re, t.im, t.im); }
__device__ __forceinline__ void acc_norm(df64& acc, cx<df64> t) { acc = df_axpy2(acc, t.re, t.re, t.im, t.im); }
// a norm that only feeds a threshold test (the serious-breakdown test of two-sided
// Lanczos): float accumulation of the high words, double in the FP64 mode
__device__ __forceinline__ void acc_norm_lo(double& acc, cx<double> t) { acc_norm(acc, t); }
__device__ __forceinline__ void acc_norm_lo(float& acc, cx<float> t) { acc = fmaf(t.re, t.re, fmaf(t.im, t.im, acc)); }
__device__ __forceinline__ void acc_norm_lo(float& acc, cx<df64> t) {
  acc = fmaf(t.re.hi, t.re.hi, fmaf(t.im.hi, t.im.hi, acc));
}
template <class A> struct NormLo { using T = float; };
template <> struct NormLo<double> { using T = double; };
__device__ __forceinline__ double to_acc(double a, double) { return a; }
__device__ __forceinline__ df64 to_acc(float a, df64) { return {a, 0.f}; }

// accumulator += c * v  (c in accumulator type, v in vector type)
__device__ __forceinline__ void acc_axpy(cx<double>& y, cx<double> c, cx<double> v) { y = y + cmul(c, v); }
__device__ __forceinline__ void acc_axpy(cx<df64>& y, cx<df64> c, cx<float> v) { y = y + lcmul<df64, float>(v, c); }
__device__ __forceinline__ void acc_axpy(cx<df64>& y, cx<df64> c, cx<df64> v) { y = y + cmul(c, v); }

__device__ __forceinline__ cx<double> acc_to_cd(cx<double> a) { return a; }
__device__ __forceinline__ cx<double> acc_to_cd(cx<df64> a) { return {df_to_double(a.re), df_to_double(a.im)}; }
__device__ __forceinline__ cx<double> vec_to_cd(cx<double> a) { return a; }
__device__ __forceinline__ cx<double> vec_to_cd(cx<float> a) { return {(double)a.re, (double)a.im}; }
__device__ __forceinline__ cx<double> vec_to_cd(cx<df64> a) { return {df_to_double(a.re), df_to_double(a.im)}; }

template <class R> __device__ __forceinline__ cx<R> cd_to(double re, double im) {
  return {from_double<R>(re), from_double<R>(im)};
}

void split_const(double d, float hl[2]) {
  hl[0] = (float)d;
  hl[1] = (float)(d - (double)hl[0]);
}
// a constant from its double value and its host-side float split (no device FP64 work)
__device__ __forceinline__ double hconst(double, double d, const float*) { return d; }
__device__ __forceinline__ float hconst(float, double, const float* hl) { return hl[0]; }
__device__ __forceinline__ df64 hconst(df64, double, const float* hl) { return {hl[0], hl[1]}; }

// step scalars: slot q of RHS r
template <class P>
__device__ __forceinline__ cx<typename P::R> ld_scal(const void* scal, int r, int q) {
  return ld_vec((const typename P::vec_t*)scal + (size_t)r * 8 + q);
}
template <class P>
__device__ __forceinline__ void st_scal(void* scal, int r, int q, double re, double im) {
  st_vec((typename P::vec_t*)scal + (size_t)r * 8 + q, cd_to<typename P::R>(re, im));
}
// scalars of step j from its coefficients nv_j, gamma_j, nw_j, beta_j and the previous
// normalisations nv_{j-1}, nw_{j-1} (run by one thread):
//   1/nv_j, gamma_j/nv_{j-1}, 1/conj(nw_j), conj(beta_j)/conj(nw_{j-1})
template <class P>
__device__ __forceinline__ void set_step_scal(void* scal, int r, double nv, double2 gam, double2 nw, double2 bet,
                                              double nvp, double2 nwp) {
  st_scal<P>(scal, r, 0, 1.0 / nv, 0.0);
  st_scal<P>(scal, r, 1, gam.x / nvp, gam.y / nvp);
  const double den = nw.x * nw.x + nw.y * nw.y;
  st_scal<P>(scal, r, 2, nw.x / den, nw.y / den);  // 1/conj(nw) = nw/|nw|^2
  // conj(beta)/conj(nwp) = conj(beta/nwp), beta/nwp = beta conj(nwp)/|nwp|^2
  const double dp = nwp.x * nwp.x + nwp.y * nwp.y;
  const double qr = (bet.x * nwp.x + bet.y * nwp.y) / dp, qi = (bet.y * nwp.x - bet.x * nwp.y) / dp;
  st_scal<P>(scal, r, 3, qr, -qi);
}

// ------------------------------------------------------------ block reductions
// Each thread passes its values; the block's sums go to partials[(part0 + bx)*4 + q]
// (part0: the problem's first slot, bx: the block's index within the problem, so the
// slots do not depend on the launch order of the blocks). Returns true in the last block
// to finish for this problem, where tot[] (valid in thread 0) holds the fixed-order total
// over all its blocks.
// The block's per-warp sums (thread 0 adds them in warp order).
template <int NQ, int BS>
__device__ __forceinline__ void block_sums(const double (&v)[NQ], double (&bsum)[NQ]) {
  __shared__ double sred[BS / 32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double w = warp_sum(v[q]);
    if (lane == 0) sred[warp][q] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = 0.0;
      for (int w = 0; w < BS / 32; ++w) s += sred[w][q];
      bsum[q] = s;
    }
  }
}
// Double-float values: warp sums and the sum over warps stay in float pairs (float
// pipes); thread 0 converts the block's sums to double once.
template <int NQ, int BS>
__device__ __forceinline__ void block_sums(const df64 (&v)[NQ], double (&bsum)[NQ]) {
  __shared__ float2 sdf[BS / 32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const df64 w = warp_sum(v[q]);
    if (lane == 0) sdf[warp][q] = make_float2(w.hi, w.lo);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      df64 s = df_zero();
      for (int w = 0; w < BS / 32; ++w) s = s + df64{sdf[w][q].x, sdf[w][q].y};
      bsum[q] = df_to_double(s);
    }
  }
}

template <int NQ, int BS, class T>
__device__ __forceinline__ bool reduce_last(T (&v)[NQ], double* partials, unsigned* counters, int r, int part0,
                                            int bx, int nblk, double (&tot)[NQ]) {
  __shared__ double sred[BS / 32][4];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double bsum[NQ];
  block_sums<NQ, BS>(v, bsum);
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) partials[(size_t)(part0 + bx) * 4 + q] = bsum[q];
    __threadfence();
    unsigned prev = atomicAdd(&counters[r], 1u);
    s_last = (prev == (unsigned)(nblk - 1));
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double loc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) loc[q] = 0.0;
  for (int b = tid; b < nblk; b += BS) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) loc[q] += __ldcg(&partials[(size_t)(part0 + b) * 4 + q]);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double w = warp_sum(loc[q]);
    if (lane == 0) sred[warp][q] = w;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = 0.0;
      for (int w = 0; w < BS / 32; ++w) s += sred[w][q];
      tot[q] = s;
    }
    counters[r] = 0u;
  }
  return true;
}

// the site of this thread: problem r (from the block map), its descriptor, block within it
struct SiteRef {
  int r, bx, s;
  bool active;
  const ProbDesc* d;
};
// rev = true: the block map walked backwards (the vector update), so that an update starts
// where the preceding step ended and the next step where the update ended: the tail of what
// one kernel wrote is still in L2 when the next kernel reads it first
template <int BS, bool rev = false>
__device__ __forceinline__ SiteRef site_ref(const Batch& b) {
  const int2 m = __ldg(&b.blk_map[rev ? b.nblocks - 1 - (int)blockIdx.x : (int)blockIdx.x]);
  const int r = m.x;
  const ProbDesc* d = &b.desc[r];
  const int bx = m.y;
  const int s = bx * BS + threadIdx.x;
  return {r, bx, s, s < d->g.V, d};
}


// ------------------------------------------------------------ pack / unpack
template <class P, int BS>
__global__ void __launch_bounds__(BS) k_pack(Batch bt, const double2* __restrict__ x, typename P::vec_t* xi,
                                                 typename P::vec_t* xi2, Coefs c, double* partials,
                                                 unsigned* counters, int want_norm, void* scal) {
  using R = typename P::R;
  const SiteRef sr = site_ref<BS>(bt);
  const int s = sr.s, r = sr.r;
  const int V = sr.d->g.V;
  const size_t voff = sr.d->voff;
  double n2 = 0.0;
  if (sr.active) {
    const double2* src = x + voff + (size_t)s * 12;
    typename P::vec_t* dst = xi + voff + s;
    typename P::vec_t* dst2 = xi2 ? xi2 + voff + s : nullptr;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 z = src[k];
      n2 = fma(z.x, z.x, fma(z.y, z.y, n2));
      st_vec(dst + (size_t)k * V, cd_to<R>(z.x, z.y));
      if (dst2) st_vec(dst2 + (size_t)k * V, cd_to<R>(z.x, z.y));
    }
  }
  if (!want_norm) return;
  double v[1] = {n2}, tot[1];
  if (reduce_last<1, BS>(v, partials, counters, r, sr.d->block0, sr.bx, sr.d->nblk, tot) && threadIdx.x == 0) {
    double nrm = sqrt(tot[0]);
    size_t o = (size_t)r * c.ld + 1;
    c.nv[o] = nrm > 0.0 ? nrm : 1.0;
    c.nw[o] = make_double2(nrm > 0.0 ? nrm : 1.0, 0.0);
    c.bet[o] = make_double2(0.0, 0.0);
    c.gam[o] = make_double2(0.0, 0.0);
    c.status[r] = nrm > 0.0 ? kStOK : kStZero;
    c.kbreak[r] = 0;
    if (scal) set_step_scal<P>(scal, r, c.nv[o], c.gam[o], c.nw[o], c.bet[o], 1.0, make_double2(1.0, 0.0));
  }
}

template <class P, int BS>
__global__ void __launch_bounds__(BS) k_unpack(Batch bt, const typename P::vec_t* __restrict__ xi, double2* y) {
  const SiteRef sr = site_ref<BS>(bt);
  if (!sr.active) return;
  const int V = sr.d->g.V;
  const typename P::vec_t* src = xi + sr.d->voff + sr.s;
  double2* dst = y + sr.d->voff + (size_t)sr.s * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    cx<double> z = vec_to_cd(ld_vec(src + (size_t)k * V));
    dst[k] = make_double2(z.re, z.im);
  }
}

// ------------------------------------------------------------ the stencil
// Spin structure in the DeGrand-Rossi basis: gamma_nu = [[0, B],[B^dag, 0]] in 2x2 spin
// blocks with B_x = [[0,i],[i,0]], B_y = [[0,-1],[1,0]], B_z = [[i,0],[0,-i]], B_t = 1.
// Forward hop (1 - gamma): h = psi_u - B psi_l, result (U h, -B^dag U h).
// Backward hop (1 + gamma): h = psi_u + B psi_l, result (U^dag h, +B^dag U^dag h).
// Every entry of B and B^dag is a power of i, so (B psi_l)_s = i^q psi_{src}: the tables
// hold, per direction, the source spin and the exponent q of both components of
// B psi_l (sources are the lower spins 2, 3) and of B^dag g (sources are 0, 1).
// The eight hops run through one loop body (the double-float body is large; unrolling
// the hops overflowed the instruction cache).
__constant__ int c_bsrc[4][2] = {{3, 2}, {3, 2}, {2, 3}, {2, 3}};
__constant__ int c_bph[4][2] = {{1, 1}, {2, 0}, {1, 3}, {0, 0}};
__constant__ int c_dsrc[4][2] = {{1, 0}, {1, 0}, {0, 1}, {0, 1}};
__constant__ int c_dph[4][2] = {{3, 3}, {0, 2}, {3, 1}, {0, 0}};

__device__ __forceinline__ double rneg(double a, bool n) { return n ? -a : a; }
__device__ __forceinline__ float rneg(float a, bool n) { return n ? -a : a; }
__device__ __forceinline__ df64 rneg(df64 a, bool n) { return n ? df64{-a.hi, -a.lo} : a; }
// i^q z
template <class R> __device__ __forceinline__ cx<R> rot(cx<R> z, int q) {
  const bool sw = q & 1;
  cx<R> r = {sw ? z.im : z.re, sw ? z.re : z.im};
  return {rneg(r.re, q == 1 || q == 2), rneg(r.im, q >= 2)};
}
// cos(q pi/2), sin(q pi/2) and z + i^q w with them (see hopping_plain)
template <class R> __device__ __forceinline__ R phase_c(int q) { return R((q == 0) - (q == 2)); }
template <class R> __device__ __forceinline__ R phase_s(int q) { return R((q == 1) - (q == 3)); }
__device__ __forceinline__ cx<float> add_rot(cx<float> z, cx<float> w, float c, float s) {
  return {__fmaf_rn(-s, w.im, __fmaf_rn(c, w.re, z.re)), __fmaf_rn(s, w.re, __fmaf_rn(c, w.im, z.im))};
}
__device__ __forceinline__ cx<double> add_rot(cx<double> z, cx<double> w, double c, double s) {
  return {__fma_rn(-s, w.im, __fma_rn(c, w.re, z.re)), __fma_rn(s, w.re, __fma_rn(c, w.im, z.im))};
}
__device__ __forceinline__ cx<double> lconj(cx<double> u, bool c) { return {u.re, c ? -u.im : u.im}; }
__device__ __forceinline__ cx<float> lconj(cx<float> u, bool c) { return {u.re, c ? -u.im : u.im}; }

__device__ __forceinline__ void site_coords(const Geometry& g, int s, int& x, int& y, int& z, int& t) {
  x = s % g.Lx;
  int q = s / g.Lx;
  y = q % g.Ly;
  q /= g.Ly;
  z = q % g.Lz;
  t = q / g.Lz;
}

__device__ __forceinline__ void hopping_df(cx<df64> (&accn)[12], const float4* __restrict__ src,
                                           const float2* __restrict__ links, const Geometry& g, int s,
                                           const int (&xc)[4], df64 ef, df64 eb);

// vector element for the hopping sum: as stored, or the high words of a float pair
__device__ __forceinline__ cx<double> ld_hop(const double2* p) { return ld_vec(p); }
__device__ __forceinline__ cx<float> ld_hop(const float2* p) { return ld_vec(p); }
__device__ __forceinline__ cx<float> ld_hop(const float4* p) {
  const float4 v = *p;
  return {v.x, v.z};
}

// acc = sum over the 8 hops of the hopping term for source `src` at site s in arithmetic
// R with links of type L; ef / eb multiply the forward / backward t hops (e^{+-mu}).
template <class R, class L, class VT, class LT>
__device__ __forceinline__ void hopping_plain(cx<R> (&acc)[12], const VT* __restrict__ src,
                                              const LT* __restrict__ links, const Geometry& g, int s,
                                              const int (&xc)[4], R ef, R eb) {
  const int V = g.V;
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = czero<R>();
#pragma unroll 1
  for (int hop = 0; hop < 8; ++hop) {
    const int nu = hop >> 1;
    const bool fwd = (hop & 1) == 0;
    const int Ln = nu == 0 ? g.Lx : (nu == 1 ? g.Ly : (nu == 2 ? g.Lz : g.Lt));
    const int st = nu == 0 ? 1 : (nu == 1 ? g.Lx : (nu == 2 ? g.Lx * g.Ly : g.Lx * g.Ly * g.Lz));
    const int c = xc[0] * (nu == 0) + xc[1] * (nu == 1) + xc[2] * (nu == 2) + xc[3] * (nu == 3);
    const int sn = fwd ? (c == Ln - 1 ? s - (Ln - 1) * st : s + st) : (c == 0 ? s + (Ln - 1) * st : s - st);
    const int ls = fwd ? s : sn;
    // link: U_nu(s) forward, U_nu(s - nu)^dag backward
    cx<L> u[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const int idx = fwd ? e : (e % 3) * 3 + e / 3;
      u[e] = lconj(ld_link(links + (size_t)(nu * 9 + idx) * V + ls), !fwd);
    }
    const int b0s = c_bsrc[nu][0], b1s = c_bsrc[nu][1];
    const int b0q = (c_bph[nu][0] + (fwd ? 2 : 0)) & 3, b1q = (c_bph[nu][1] + (fwd ? 2 : 0)) & 3;
    // i^q as (c, s) in {0, +-1}: z + i^q w = (z.re + c w.re - s w.im, z.im + c w.im + s w.re)
    // by fused multiply-adds; one of c, s is zero, so each component is rounded once, as a
    // plain addition of the rotated term would be
    const R c0 = phase_c<R>(b0q), s0 = phase_s<R>(b0q), c1 = phase_c<R>(b1q), s1 = phase_s<R>(b1q);
    cx<R> h0[3], h1[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      const cx<R> p0 = ld_hop(src + (size_t)(0 + col) * V + sn);
      const cx<R> p1 = ld_hop(src + (size_t)(3 + col) * V + sn);
      const cx<R> q0 = ld_hop(src + (size_t)(3 * b0s + col) * V + sn);
      const cx<R> q1 = ld_hop(src + (size_t)(3 * b1s + col) * V + sn);
      h0[col] = add_rot(p0, q0, c0, s0);
      h1[col] = add_rot(p1, q1, c1, s1);
    }
    const bool sc = nu == 3;
    const R fac = fwd ? ef : eb;
    const int d0s = c_dsrc[nu][0], d1s = c_dsrc[nu][1];
    const int d0q = (c_dph[nu][0] + (fwd ? 2 : 0)) & 3, d1q = (c_dph[nu][1] + (fwd ? 2 : 0)) & 3;
    const R e0 = phase_c<R>(d0q), f0 = phase_s<R>(d0q), e1 = phase_c<R>(d1q), f1 = phase_s<R>(d1q);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cx<R> g0 = lcmul<R, L>(u[a * 3 + 0], h0[0]) + lcmul<R, L>(u[a * 3 + 1], h0[1]) + lcmul<R, L>(u[a * 3 + 2], h0[2]);
      cx<R> g1 = lcmul<R, L>(u[a * 3 + 0], h1[0]) + lcmul<R, L>(u[a * 3 + 1], h1[1]) + lcmul<R, L>(u[a * 3 + 2], h1[2]);
      if (sc) {
        g0 = cscale(g0, fac);
        g1 = cscale(g1, fac);
      }
      acc[0 + a] = acc[0 + a] + g0;
      acc[3 + a] = acc[3 + a] + g1;
      acc[6 + a] = add_rot(acc[6 + a], d0s == 0 ? g0 : g1, e0, f0);
      acc[9 + a] = add_rot(acc[9 + a], d1s == 0 ? g0 : g1, e1, f1);
    }
  }
}

template <class P>
__device__ __forceinline__ void hopping(cx<typename P::R> (&acc)[12], const typename P::vec_t* __restrict__ src,
                                        const typename P::link_t* __restrict__ links, const Geometry& g, int s,
                                        const int (&xc)[4], typename P::R ef, typename P::R eb) {
  if constexpr (P::id == PrecDF64::id) {
    hopping_df(acc, src, links, g, s, xc, ef, eb);
  } else if constexpr (P::id == PrecDF64R::id) {
    cx<float> af[12];
    hopping_plain<float, float>(af, src, links, g, s, xc, ef.hi, eb.hi);
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {{af[k].re, 0.f}, {af[k].im, 0.f}};
  } else {
    hopping_plain<typename P::R, typename P::L>(acc, src, links, g, s, xc, ef, eb);
  }
}

// ---- double-float hopping in compensated form -------------------------------------------
// The links are double-float too: a plane of float hi parts and, 36 V elements further on,
// a plane of lo parts (|lo| <= 2^-24 |hi|). The products U_ab h_b are summed as in the
// compensated dot product of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26 (2005), "Dot2"):
// the product of U.hi with h.hi is exact as (p, e) (p = U.hi*h.hi, e = fma(U.hi, h.hi, -p)),
// U.hi*h.lo is folded into e with one FMA, the running sum takes p through TwoSum, and all
// error terms are accumulated in the low word without renormalising; U.lo*h.hi, a term of
// relative size 2^-24, is added to the low word in plain float arithmetic once per row
// (the lo links are loaded with the hi links at the start of the hop).
// Sums are renormalised once, when the hopping term is complete. Error: a few units of
// 2^-48 relative to the summed magnitudes, as for the normalised pair arithmetic.
struct dfu {  // unnormalised pair: value hi + lo
  float hi, lo;
};
__device__ __forceinline__ void madd_u(dfu& acc, float u, df64 h) {
  const float p = __fmul_rn(u, h.hi);
  float e = __fmaf_rn(u, h.hi, -p);
  e = __fmaf_rn(u, h.lo, e);
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, err));
}
// acc = u h, exactly as (p, e)
__device__ __forceinline__ void set_u(dfu& acc, float u, df64 h) {
  const float p = __fmul_rn(u, h.hi);
  float e = __fmaf_rn(u, h.hi, -p);
  acc = {p, __fmaf_rn(u, h.lo, e)};
}
__device__ __forceinline__ dfu add_u(dfu a, dfu b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return {s, __fadd_rn(__fadd_rn(a.lo, b.lo), err)};
}
__device__ __forceinline__ dfu neg_u(dfu a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df64 norm_u(dfu a) { return df_fast_two_sum(a.hi, a.lo); }
__device__ __forceinline__ dfu to_u(df64 a) { return {a.hi, a.lo}; }
struct cxu {
  dfu re, im;
};
__device__ __forceinline__ cxu cadd_u(cxu a, cxu b) { return {add_u(a.re, b.re), add_u(a.im, b.im)}; }
// i^q z
__device__ __forceinline__ cxu rot_u(cxu z, int q) {
  const bool sw = q & 1;
  cxu r = {sw ? z.im : z.re, sw ? z.re : z.im};
  const bool nre = q == 1 || q == 2, nim = q >= 2;
  return {nre ? neg_u(r.re) : r.re, nim ? neg_u(r.im) : r.im};
}

__device__ __forceinline__ void hopping_df(cx<df64> (&accn)[12], const float4* __restrict__ src,
                                           const float2* __restrict__ links, const Geometry& g, int s,
                                           const int (&xc)[4], df64 ef, df64 eb) {
  const int V = g.V;
  const float2* __restrict__ links_lo = links + (size_t)36 * V;
  cxu acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 1
  for (int hop = 0; hop < 8; ++hop) {
    const int nu = hop >> 1;
    const bool fwd = (hop & 1) == 0;
    const int Ln = nu == 0 ? g.Lx : (nu == 1 ? g.Ly : (nu == 2 ? g.Lz : g.Lt));
    const int st = nu == 0 ? 1 : (nu == 1 ? g.Lx : (nu == 2 ? g.Lx * g.Ly : g.Lx * g.Ly * g.Lz));
    const int c = xc[0] * (nu == 0) + xc[1] * (nu == 1) + xc[2] * (nu == 2) + xc[3] * (nu == 3);
    const int sn = fwd ? (c == Ln - 1 ? s - (Ln - 1) * st : s + st) : (c == 0 ? s + (Ln - 1) * st : s - st);
    const int ls = fwd ? s : sn;
    cx<float> u[9], ulo[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const int idx = fwd ? e : (e % 3) * 3 + e / 3;
      u[e] = lconj(ld_link(links + (size_t)(nu * 9 + idx) * V + ls), !fwd);
      ulo[e] = lconj(ld_link(links_lo + (size_t)(nu * 9 + idx) * V + ls), !fwd);
    }
    const int b0s = c_bsrc[nu][0], b1s = c_bsrc[nu][1];
    const int b0q = (c_bph[nu][0] + (fwd ? 2 : 0)) & 3, b1q = (c_bph[nu][1] + (fwd ? 2 : 0)) & 3;
    cx<df64> h0[3], h1[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      const cx<df64> p0 = ld_vec(src + (size_t)(0 + col) * V + sn);
      const cx<df64> p1 = ld_vec(src + (size_t)(3 + col) * V + sn);
      const cx<df64> q0 = rot(ld_vec(src + (size_t)(3 * b0s + col) * V + sn), b0q);
      const cx<df64> q1 = rot(ld_vec(src + (size_t)(3 * b1s + col) * V + sn), b1q);
      // projections, unnormalised (their low words only enter through FMAs below)
      const dfu r0 = add_u(to_u(p0.re), to_u(q0.re)), i0 = add_u(to_u(p0.im), to_u(q0.im));
      const dfu r1 = add_u(to_u(p1.re), to_u(q1.re)), i1 = add_u(to_u(p1.im), to_u(q1.im));
      h0[col] = {{r0.hi, r0.lo}, {i0.hi, i0.lo}};
      h1[col] = {{r1.hi, r1.lo}, {i1.hi, i1.lo}};
    }
    const bool sc = nu == 3;
    const df64 fac = fwd ? ef : eb;
    const int d0s = c_dsrc[nu][0], d1s = c_dsrc[nu][1];
    const int d0q = (c_dph[nu][0] + (fwd ? 2 : 0)) & 3, d1q = (c_dph[nu][1] + (fwd ? 2 : 0)) & 3;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cxu g0, g1;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const cx<float> ub = u[a * 3 + b];
        // (u.re + i u.im)(h.re + i h.im); the first product of each sum sets it
        if (b == 0) {
          set_u(g0.re, ub.re, h0[b].re);
          set_u(g0.im, ub.re, h0[b].im);
          set_u(g1.re, ub.re, h1[b].re);
          set_u(g1.im, ub.re, h1[b].im);
        } else {
          madd_u(g0.re, ub.re, h0[b].re);
          madd_u(g0.im, ub.re, h0[b].im);
          madd_u(g1.re, ub.re, h1[b].re);
          madd_u(g1.im, ub.re, h1[b].im);
        }
        madd_u(g0.re, -ub.im, h0[b].im);
        madd_u(g0.im, ub.im, h0[b].re);
        madd_u(g1.re, -ub.im, h1[b].im);
        madd_u(g1.im, ub.im, h1[b].re);
      }
      // U.lo row a times h.hi, into the low words
      float c0r = 0.f, c0i = 0.f, c1r = 0.f, c1i = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const cx<float> ul = ulo[a * 3 + b];
        c0r = __fmaf_rn(ul.re, h0[b].re.hi, __fmaf_rn(-ul.im, h0[b].im.hi, c0r));
        c0i = __fmaf_rn(ul.re, h0[b].im.hi, __fmaf_rn(ul.im, h0[b].re.hi, c0i));
        c1r = __fmaf_rn(ul.re, h1[b].re.hi, __fmaf_rn(-ul.im, h1[b].im.hi, c1r));
        c1i = __fmaf_rn(ul.re, h1[b].im.hi, __fmaf_rn(ul.im, h1[b].re.hi, c1i));
      }
      g0.re.lo = __fadd_rn(g0.re.lo, c0r);
      g0.im.lo = __fadd_rn(g0.im.lo, c0i);
      g1.re.lo = __fadd_rn(g1.re.lo, c1r);
      g1.im.lo = __fadd_rn(g1.im.lo, c1i);
      if (sc) {
        const cx<df64> n0 = cscale(cx<df64>{norm_u(g0.re), norm_u(g0.im)}, fac);
        const cx<df64> n1 = cscale(cx<df64>{norm_u(g1.re), norm_u(g1.im)}, fac);
        g0 = {to_u(n0.re), to_u(n0.im)};
        g1 = {to_u(n1.re), to_u(n1.im)};
      }
      acc[0 + a] = cadd_u(acc[0 + a], g0);
      acc[3 + a] = cadd_u(acc[3 + a], g1);
      acc[6 + a] = cadd_u(acc[6 + a], rot_u(d0s == 0 ? g0 : g1, d0q));
      acc[9 + a] = cadd_u(acc[9 + a], rot_u(d1s == 0 ? g0 : g1, d1q));
    }
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) accn[k] = {norm_u(acc[k].re), norm_u(acc[k].im)};
}

// (gamma5 D psi)_k at the centre site from the hopping sum: mass*psi - hop/2, lower spins negated.
template <class R>
__device__ __forceinline__ cx<R> g5d(int k, cx<R> psi, cx<R> hk, R mass) {
  cx<R> d = cscale(psi, mass) - chalf(hk);
  return k >= 6 ? -d : d;
}
__device__ __forceinline__ cx<df64> g5d(int k, cx<df64> psi, cx<df64> hk, df64 mass) {
  const cx<df64> d = {df_axpy1(-df_half(hk.re), mass, psi.re), df_axpy1(-df_half(hk.im), mass, psi.im)};
  return k >= 6 ? -d : d;
}

// ---- the recurrence at one site: scalars real (RS, RC) or complex -----------------------
// In the recurrences 1/nv_j and beta_j are real, gamma_j and 1/conj(nw_j) complex: side v of
// two-sided Lanczos scales by a real and subtracts a complex multiple, side w the reverse,
// Lanczos has both real.
template <bool RS, class R>
__device__ __forceinline__ cx<R> smul(cx<R> s, cx<R> z) {
  return RS ? cscale(z, s.re) : cmul(s, z);
}
template <bool RS>
__device__ __forceinline__ cx<df64> smul(cx<df64> s, cx<df64> z) {
  if (RS) return {z.re * s.re, z.im * s.re};
  return {df_axpy2(df_zero(), s.re, z.re, -s.im, z.im), df_axpy2(df_zero(), s.re, z.im, s.im, z.re)};
}
// s q - c w
template <bool RS, bool RC, class R>
__device__ __forceinline__ cx<R> smulsub(cx<R> s, cx<R> q, cx<R> c, cx<R> w) {
  return smul<RS>(s, q) - smul<RC>(c, w);
}
template <bool RS, bool RC>
__device__ __forceinline__ cx<df64> smulsub(cx<df64> s, cx<df64> q, cx<df64> c, cx<df64> w) {
  if (RS && RC) return {df_axpy2(df_zero(), s.re, q.re, -c.re, w.re), df_axpy2(df_zero(), s.re, q.im, -c.re, w.im)};
  if (RS) return {df_axpy2(q.re * s.re, -c.re, w.re, c.im, w.im), df_axpy2(q.im * s.re, -c.re, w.im, -c.im, w.re)};
  if (RC)
    return {df_axpy2(-(w.re * c.re), s.re, q.re, -s.im, q.im), df_axpy2(-(w.im * c.re), s.re, q.im, s.im, q.re)};
  // both complex: each component one compensated four-term sum
  return {df_dot4(s.re, q.re, -s.im, q.im, -c.re, w.re, c.im, w.im),
          df_dot4(s.re, q.im, s.im, q.re, -c.re, w.im, -c.im, w.re)};
}
// out = scl (gamma5 D t_j) - cf t_{j-1} at one site, 12 components, with t_j the
// unnormalised current vector (psi) and t_{j-1} the previous one; the alpha partial: Lanczos
// t_j^dag out, two-sided side w: tw_j^dag p (p from side v); the finaliser divides by the
// normalisation
template <bool RS, bool RC, int DOT, class R, class VT, class AT>
__device__ __forceinline__ void step_site(const VT* src, const VT* prv, VT* out, const VT* pp, int V, int s,
                                          cx<R> scl, cx<R> cf, const cx<R> (&acc)[12], R mass, cx<AT>& dot) {
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const cx<R> psi = ld_vec(src + (size_t)k * V + s);
    const cx<R> ok = smulsub<RS, RC>(scl, g5d(k, psi, acc[k], mass), cf, ld_vec(prv + (size_t)k * V));
    st_vec(out + (size_t)k * V, ok);
    if (DOT == 1) acc_dot(dot, psi, ok);
    if (DOT == 2) acc_dot(dot, psi, ld_vec(pp + (size_t)k * V));
  }
}

// the step index and the step's vectors (device-side state or host fields): t_j, t_{j-1},
// the destination of t_{j+1}, and the same three on the w side
struct StepPtrs {
  int j;
  const void* tc;
  const void* tp;
  void* tn;
  const void* wc;
  const void* wp;
  void* wn;
};
__device__ __forceinline__ StepPtrs step_ptrs(const StepArgs& a) {
  if (!a.jdev) return {a.j, a.tc, a.tp, a.tn, nullptr, nullptr, nullptr};
  const int j = __ldcg(a.jdev);
  char* vr = (char*)a.vring;
  char* wr = (char*)a.wring;
  const size_t pb = a.pool_bytes;
  char* wc = wr + pb * (j & 1);
  char* wp = wr + pb * ((j - 1) & 1);
  if (a.slot_tab) {
    // stored basis: slot i holds t_{i+1}; t_0 is the zeroed ring slot 0
    const void* tp = j == 1 ? (const void*)vr : (const void*)a.slot_tab[j - 2];
    return {j, a.slot_tab[j - 1], tp, a.slot_tab[j], wc, wp, wp};
  }
  char* tc = vr + pb * (j & 1);
  char* tp = vr + pb * ((j - 1) & 1);
  return {j, tc, tp, tp, wc, wp, wp};
}

// Register caps of the step kernels (the warps they add hide the load latency at the start
// of each hop; measured at 16^4 with 12 right-hand sides): 128 registers a thread for the
// strict double-float step (16 warps an SM; its hop body fits, tighter caps spill hundreds
// of bytes and run slower), 85 for the relaxed step (24 warps; it fits in 80: 0.50 ->
// 0.46 ms) and 64 for the float step (32 warps, a few spilled words: 0.32 -> 0.27 ms).
// FP64 keeps the compiler's choice.
// Resident threads per SM each step kernel is compiled for (the register cap follows:
// 65536 / threads); overridable at build time to measure other splits.
#ifndef OV_STEP_THREADS_DF64
#define OV_STEP_THREADS_DF64 512
#endif
#ifndef OV_STEP_THREADS_DF64R
#define OV_STEP_THREADS_DF64R 768
#endif
#ifndef OV_STEP_THREADS_F32
#define OV_STEP_THREADS_F32 1024
#endif
template <class P, int BS>
constexpr int step_min_blocks() {
  constexpr int t = P::id == PrecDF64::id    ? OV_STEP_THREADS_DF64
                    : P::id == PrecDF64R::id ? OV_STEP_THREADS_DF64R
                    : P::id == PrecF32::id   ? OV_STEP_THREADS_F32
                                             : BS;
  return t / BS > 0 ? t / BS : 1;
}

template <class P, int MODE, int BS>
__global__ void __launch_bounds__(BS, step_min_blocks<P, BS>()) k_step(StepArgs a) {
  using R = typename P::R;
  using V_t = typename P::vec_t;
  using L_t = typename P::link_t;
  using A = typename P::A;
  using AT = typename AccOf<P>::A;
  using AS = typename AccOf<P>::st;
  const SiteRef sr = site_ref<BS>(a.b);
  const ProbDesc& d = *sr.d;
  const Geometry g = d.g;
  const int s = sr.s, r = sr.r;
  const bool active = sr.active;
  const int ss = active ? s : 0;
  const size_t vo = d.voff;
  const L_t* links = (const L_t*)d.links;
  const R mass = hconst(R(), d.mass, d.mass_hl);
  const R emu = hconst(R(), d.emu, d.emu_hl), emui = hconst(R(), d.emui, d.emui_hl);
  const StepPtrs sp = step_ptrs(a);
  const size_t co = (size_t)r * a.c.ld + sp.j;
  int xc[4];
  site_coords(g, ss, xc[0], xc[1], xc[2], xc[3]);

  cx<A> dot = {rzero<A>(), rzero<A>()};
  cx<R> acc[12];

  if (MODE == kModeApply) {
    if (active) {
      const V_t* tv = (const V_t*)a.tv + vo;
      hopping<P>(acc, tv, links, g, s, xc, a.dagger ? emui : emu, a.dagger ? emu : emui);
      V_t* out = (V_t*)a.p + vo + s;
#pragma unroll
      for (int k = 0; k < 12; ++k) st_vec(out + (size_t)k * g.V, g5d(k, ld_vec(tv + (size_t)k * g.V + s), acc[k], mass));
    }
    return;
  }

  const V_t* tc = (const V_t*)sp.tc + vo;
  if (MODE == kModeRegen) {
    // second pass, all coefficients known: p = A t_j / nv_j - (gamma_j / nv_{j-1}) t_{j-1},
    // t_{j+1} = p - (alpha_j / nv_j) t_j (over t_{j-1}: each thread reads its own entry of
    // t_{j-1} before writing it), and y += (c_j / nv_j) t_j
    if (!active) return;
    const double nvj = a.c.nv[co];
    const double nvp = sp.j > 1 ? a.c.nv[co - 1] : 1.0;
    const R rinv = from_double<R>(1.0 / nvj);
    const double2 gj = a.c.gam[co];
    const cx<R> cg = cd_to<R>(gj.x / nvp, gj.y / nvp);
    const double2 aj = a.c.alp[co];
    const cx<R> ca = cd_to<R>(aj.x / nvj, aj.y / nvj);
    hopping<P>(acc, tc, links, g, s, xc, emu, emui);
    const V_t* tp = (const V_t*)sp.tp + vo + s;
    V_t* tn = (V_t*)sp.tn + vo + s;
    const cx<AT> cjv = ld_acc((const AS*)a.cacc + (size_t)r * a.c.ld + sp.j);
    AS* ya = (AS*)a.yacc + vo + s;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const cx<R> psi = ld_vec(tc + (size_t)k * g.V + s);
      const cx<R> pk = cscale(g5d(k, psi, acc[k], mass), rinv) - cmul(cg, ld_vec(tp + (size_t)k * g.V));
      st_vec(tn + (size_t)k * g.V, pk - cmul(ca, psi));
      cx<AT> y = ld_acc(ya + (size_t)k * g.V);
      acc_axpy(y, cjv, psi);
      st_acc(ya + (size_t)k * g.V, y);
    }
    return;
  }

  // Lanczos: one side (v). Two-sided: side 0 is v with A, side 1 is w with A^dag.
  //   p = A t_j / nv_j - (gamma_j / nv_{j-1}) t_{j-1}
  //   r = A^dag tw_j / conj(nw_j) - (conj(beta_j) / conj(nw_{j-1})) tw_{j-1}
  //   alpha_j = t_j^dag p / nv_j (Lanczos) or tw_j^dag p / nw_j (two-sided)
  const int nsides = MODE == kModeTwoSided ? 2 : 1;
#pragma unroll 1
  for (int side = 0; side < nsides; ++side) {
    const cx<R> scl = ld_scal<P>(a.scal, r, 2 * side);
    const cx<R> cf = ld_scal<P>(a.scal, r, 2 * side + 1);
    if (active) {
      const V_t* src = side == 0 ? tc : (const V_t*)sp.wc + vo;
      hopping<P>(acc, src, links, g, s, xc, side == 0 ? emu : emui, side == 0 ? emui : emu);
      const V_t* prv = side == 0 ? (const V_t*)sp.tp + vo + s : (const V_t*)sp.wp + vo + s;
      V_t* out = side == 0 ? (V_t*)a.p + vo + s : (V_t*)a.r + vo + s;
      const V_t* pp = (const V_t*)a.p + vo + s;
      if (MODE == kModeLanczos)
        step_site<true, true, 1>(src, prv, out, pp, g.V, s, scl, cf, acc, mass, dot);
      else if (side == 0)
        step_site<true, false, 0>(src, prv, out, pp, g.V, s, scl, cf, acc, mass, dot);
      else
        step_site<false, false, 2>(src, prv, out, pp, g.V, s, scl, cf, acc, mass, dot);
    }
  }
  A v2[2] = {dot.re, dot.im};
  double tot[2];
  if (reduce_last<2, BS>(v2, a.partials, a.counters, r, d.block0, sr.bx, d.nblk, tot) && threadIdx.x == 0) {
    const double nvj = a.c.nv[co];
    double ar, ai;
    double2 nw = a.c.nw[co];
    if (MODE == kModeLanczos) {
      ar = tot[0] / nvj;
      ai = 0.0;
      nw = make_double2(nvj, 0.0);
    } else {
      // (tot) / nw_j
      const double den = nw.x * nw.x + nw.y * nw.y;
      ar = (tot[0] * nw.x + tot[1] * nw.y) / den;
      ai = (tot[1] * nw.x - tot[0] * nw.y) / den;
    }
    a.c.alp[co] = make_double2(ar, ai);
    // alpha_j / nv_j and conj(alpha_j) / conj(nw_j) = conj(alpha_j / nw_j)
    st_scal<P>(a.scal, r, 4, ar / nvj, ai / nvj);
    const double dw = nw.x * nw.x + nw.y * nw.y;
    st_scal<P>(a.scal, r, 5, (ar * nw.x + ai * nw.y) / dw, -((ai * nw.x - ar * nw.y) / dw));
  }
}

// ------------------------------------------------------------ vector update
// resident threads per SM the update kernel is compiled for (0: the compiler's choice, 56
// registers). 1280 (48 registers, five blocks of 256) measured 0.168 -> 0.161 ms for the
// double-float two-sided update at 16^4 x 12; 1536 spills, and 256 (145 registers, the
// loads of all twelve components in flight in one thread) runs at 0.29 ms.
#ifndef OV_UPDATE_THREADS
#define OV_UPDATE_THREADS 1280
#endif
#if OV_UPDATE_THREADS > 0
#define OV_UPDATE_BOUNDS(BS) __launch_bounds__(BS, (OV_UPDATE_THREADS / BS > 0 ? OV_UPDATE_THREADS / BS : 1))
#else
#define OV_UPDATE_BOUNDS(BS) __launch_bounds__(BS)
#endif
template <class P, int MODE, int BS>
__global__ void OV_UPDATE_BOUNDS(BS) k_update(StepArgs a) {
  using R = typename P::R;
  using V_t = typename P::vec_t;
  using A = typename P::A;
  const SiteRef sr = site_ref<BS, true>(a.b);
  const Geometry g = sr.d->g;
  const int s = sr.s, r = sr.r;
  const size_t vo = sr.d->voff;
  const StepPtrs sp = step_ptrs(a);
  const size_t co = (size_t)r * a.c.ld + sp.j;
  const cx<R> alp = ld_scal<P>(a.scal, r, 4);
  const cx<R> calp = ld_scal<P>(a.scal, r, 5);
  using NL = typename NormLo<A>::T;
  cx<A> d = {rzero<A>(), rzero<A>()};
  A nvv = rzero<A>();              // ||v~||^2: beta in Lanczos
  NL nvl = NL(0), nwl = NL(0);     // ||v~||^2, ||w~||^2 for the breakdown test of 2sL
  if (sr.active) {
    // t_{j+1} = p - (alpha_j / nv_j) t_j, tw_{j+1} = r - (conj(alpha_j) / conj(nw_j)) tw_j
    const V_t* __restrict__ pp = (const V_t*)a.p + vo + s;
    const V_t* __restrict__ vc = (const V_t*)sp.tc + vo + s;
    V_t* __restrict__ tv = (V_t*)sp.tn + vo + s;  // may be t_{j-1}: the stencil no longer reads it
    if (MODE == kModeLanczos) {
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const cx<R> t = csubmul(ld_vec(pp + (size_t)k * g.V), alp, ld_vec(vc + (size_t)k * g.V));
        st_vec(tv + (size_t)k * g.V, t);
        acc_norm(nvv, t);
      }
    } else {
      const V_t* __restrict__ rr = (const V_t*)a.r + vo + s;
      const V_t* __restrict__ wc = (const V_t*)sp.wc + vo + s;
      V_t* __restrict__ tw = (V_t*)sp.wn + vo + s;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const cx<R> t = csubmul(ld_vec(pp + (size_t)k * g.V), alp, ld_vec(vc + (size_t)k * g.V));
        const cx<R> u = csubmul(ld_vec(rr + (size_t)k * g.V), calp, ld_vec(wc + (size_t)k * g.V));
        st_vec(tv + (size_t)k * g.V, t);
        st_vec(tw + (size_t)k * g.V, u);
        acc_dot(d, u, t);
        acc_norm_lo(nvl, t);
        acc_norm_lo(nwl, u);
      }
    }
  }
  if (MODE == kModeLanczos) {
    A v1[1] = {nvv};
    double tot[1];
    if (reduce_last<1, BS>(v1, a.partials, a.counters, r, sr.d->block0, sr.bx, sr.d->nblk, tot) && threadIdx.x == 0) {
      const double b = sqrt(tot[0]);
      const double bprev = fabs(a.c.bet[co].x);
      const size_t cn = co + 1;
      const bool broke = !(b > a.breakdown_tol * (fabs(a.c.alp[co].x) + bprev));
      if (broke && a.c.status[r] == kStOK) {
        a.c.status[r] = kStLucky;
        a.c.kbreak[r] = sp.j;
      }
      const bool dead = a.c.status[r] != kStOK;
      a.c.nv[cn] = dead ? 1.0 : b;
      a.c.nw[cn] = make_double2(dead ? 1.0 : b, 0.0);
      a.c.bet[cn] = make_double2(dead ? 0.0 : b, 0.0);
      a.c.gam[cn] = make_double2(dead ? 0.0 : b, 0.0);
      set_step_scal<P>(a.scal, r, a.c.nv[cn], a.c.gam[cn], a.c.nw[cn], a.c.bet[cn], a.c.nv[co], a.c.nw[co]);
    }
  } else {
    A v4[4] = {d.re, d.im, to_acc(nvl, A()), to_acc(nwl, A())};
    double tot[4];
    if (reduce_last<4, BS>(v4, a.partials, a.counters, r, sr.d->block0, sr.bx, sr.d->nblk, tot) && threadIdx.x == 0) {
      const double dre = tot[0], dim = tot[1];
      const double ad = sqrt(dre * dre + dim * dim);
      const double b = sqrt(ad);
      const size_t cn = co + 1;
      const bool broke = !(ad > a.breakdown_tol * sqrt(tot[2]) * sqrt(tot[3])) || !(b > 0.0);
      if (broke && a.c.status[r] == kStOK) {
        a.c.status[r] = kStBreakdown;
        a.c.kbreak[r] = sp.j;
      }
      const bool dead = a.c.status[r] != kStOK;
      a.c.nv[cn] = dead ? 1.0 : b;
      a.c.nw[cn] = dead ? make_double2(1.0, 0.0) : make_double2(dre / b, dim / b);
      a.c.bet[cn] = make_double2(dead ? 0.0 : b, 0.0);
      a.c.gam[cn] = dead ? make_double2(0.0, 0.0) : make_double2(dre / b, dim / b);
      set_step_scal<P>(a.scal, r, a.c.nv[cn], a.c.gam[cn], a.c.nw[cn], a.c.bet[cn], a.c.nv[co], a.c.nw[co]);
    }
  }
  // device-side step state: the last block of the launch advances j
  if (a.jdev) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned t = atomicAdd(a.gticket, 1u);
      if (t == gridDim.x - 1) {
        *a.jdev = sp.j + 1;
        *a.gticket = 0u;
        __threadfence();
      }
    }
  }
}

// ------------------------------------------------------------ recombination
template <class P, int BS>
__global__ void __launch_bounds__(BS) k_recombine(Batch bt, const void* const* __restrict__ slots,
                                                      const typename AccOf<P>::st* __restrict__ cacc, int ldc,
                                                      const int* __restrict__ kr, const double* __restrict__ scale,
                                                      const double2* __restrict__ x, int add_x, double2* y) {
  using AT = typename AccOf<P>::A;
  const SiteRef sr = site_ref<BS>(bt);
  if (!sr.active) return;
  const int s = sr.s, r = sr.r, V = sr.d->g.V;
  const size_t vo = sr.d->voff;
  cx<AT> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = czero<AT>();
  const int k_r = kr[r];
  const typename AccOf<P>::st* cr = cacc + (size_t)r * ldc;
  for (int j = 0; j < k_r; ++j) {
    const cx<AT> cj = ld_acc(cr + j + 1);
    const typename P::vec_t* vj = (const typename P::vec_t*)slots[j] + vo + s;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc_axpy(acc[k], cj, ld_vec(vj + (size_t)k * V));
  }
  const double sc = scale[r];
  double2* dst = y + vo + (size_t)s * 12;
  const double2* xs = x + vo + (size_t)s * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    cx<double> z = acc_to_cd(acc[k]);
    z.re *= sc;
    z.im *= sc;
    if (add_x) {
      const double2 xv = xs[k];
      if (k >= 6) { z.re = -z.re; z.im = -z.im; }
      z.re += xv.x;
      z.im += xv.y;
    }
    dst[k] = make_double2(z.re, z.im);
  }
}

template <class P, int BS>
__global__ void __launch_bounds__(BS) k_finish_acc(Batch bt, const typename AccOf<P>::st* __restrict__ yacc,
                                                       const double* __restrict__ scale,
                                                       const double2* __restrict__ x, int add_x, double2* y) {
  const SiteRef sr = site_ref<BS>(bt);
  if (!sr.active) return;
  const int s = sr.s, r = sr.r, V = sr.d->g.V;
  const size_t vo = sr.d->voff;
  const double sc = scale[r];
  double2* dst = y + vo + (size_t)s * 12;
  const double2* xs = x + vo + (size_t)s * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    cx<double> z = acc_to_cd(ld_acc(yacc + vo + (size_t)k * V + s));
    z.re *= sc;
    z.im *= sc;
    if (add_x) {
      const double2 xv = xs[k];
      if (k >= 6) { z.re = -z.re; z.im = -z.im; }
      z.re += xv.x;
      z.im += xv.y;
    }
    dst[k] = make_double2(z.re, z.im);
  }
}

// ------------------------------------------------------------ launchers
void fill_consts(ProbDesc& d, double m_w, double mu) {
  d.mass = m_w + 4.0;
  d.emu = exp(mu);
  d.emui = exp(-mu);
  split_const(d.mass, d.mass_hl);
  split_const(d.emu, d.emu_hl);
  split_const(d.emui, d.emui_hl);
}

#define OV_DISPATCH(prec, CALL)                      \
  switch (prec) {                                    \
    case OV_PREC_FP64: { using P = PrecF64; CALL; break; }  \
    case OV_PREC_FP32: { using P = PrecF32; CALL; break; }  \
    default: { using P = PrecDF64; CALL; break; }           \
  }
// the block size is the one the batch's block map was built with
#define OV_BS_DISPATCH(bs, CALL)                           \
  switch (bs) {                                            \
    case 64: { constexpr int BS = 64; CALL; break; }       \
    case 256: { constexpr int BS = 256; CALL; break; }     \
    default: { constexpr int BS = 128; CALL; break; }      \
  }

cudaError_t launch_pack(int prec, const Batch& b, const double2* x, void* xi, void* xi2, Coefs c, double* partials,
                        unsigned* counters, int want_norm, void* scal, cudaStream_t st) {
  OV_BS_DISPATCH(b.block, OV_DISPATCH(prec, (k_pack<P, BS><<<b.nblocks, BS, 0, st>>>(
                                                b, x, (typename P::vec_t*)xi, (typename P::vec_t*)xi2, c, partials,
                                                counters, want_norm, scal))));
  return cudaGetLastError();
}

cudaError_t launch_unpack(int prec, const Batch& b, const void* xi, double2* y, cudaStream_t st) {
  OV_BS_DISPATCH(b.block, OV_DISPATCH(prec, (k_unpack<P, BS><<<b.nblocks, BS, 0, st>>>(
                                                b, (const typename P::vec_t*)xi, y))));
  return cudaGetLastError();
}

// steps also take kPrecDF64Relaxed (the double-float storage with float hopping)
#define OV_STEP_DISPATCH(prec, CALL)                                \
  if (prec == kPrecDF64Relaxed) { using P = PrecDF64R; CALL; }      \
  else { OV_DISPATCH(prec, CALL) }

cudaError_t launch_step(int prec, int mode, const StepArgs& a, cudaStream_t st) {
  const int grid = a.b.nblocks;
  switch (mode) {
    case kModeLanczos:
      OV_BS_DISPATCH(a.b.block, OV_STEP_DISPATCH(prec, (k_step<P, kModeLanczos, BS><<<grid, BS, 0, st>>>(a))));
      break;
    case kModeTwoSided:
      OV_BS_DISPATCH(a.b.block, OV_STEP_DISPATCH(prec, (k_step<P, kModeTwoSided, BS><<<grid, BS, 0, st>>>(a))));
      break;
    case kModeRegen:
      OV_BS_DISPATCH(a.b.block, OV_STEP_DISPATCH(prec, (k_step<P, kModeRegen, BS><<<grid, BS, 0, st>>>(a))));
      break;
    default:
      OV_BS_DISPATCH(a.b.block, OV_DISPATCH(prec, (k_step<P, kModeApply, BS><<<grid, BS, 0, st>>>(a))));
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_update(int prec, int mode, const StepArgs& a, cudaStream_t st) {
  const int grid = a.b.nblocks;
  if (mode == kModeLanczos) {
    OV_BS_DISPATCH(a.b.block, OV_DISPATCH(prec, (k_update<P, kModeLanczos, BS><<<grid, BS, 0, st>>>(a))));
  } else {
    OV_BS_DISPATCH(a.b.block, OV_DISPATCH(prec, (k_update<P, kModeTwoSided, BS><<<grid, BS, 0, st>>>(a))));
  }
  return cudaGetLastError();
}

cudaError_t launch_recombine(int prec, const Batch& b, const void* const* slots, const void* cacc, int ldc,
                             const int* k_dev, const double* scale, const double2* x, int add_x, double2* y,
                             cudaStream_t st) {
  OV_BS_DISPATCH(b.block, OV_DISPATCH(prec, (k_recombine<P, BS><<<b.nblocks, BS, 0, st>>>(
                                                b, slots, (const typename AccOf<P>::st*)cacc, ldc, k_dev, scale, x,
                                                add_x, y))));
  return cudaGetLastError();
}

cudaError_t launch_finish_acc(int prec, const Batch& b, const void* yacc, const double* scale, const double2* x,
                              int add_x, double2* y, cudaStream_t st) {
  OV_BS_DISPATCH(b.block, OV_DISPATCH(prec, (k_finish_acc<P, BS><<<b.nblocks, BS, 0, st>>>(
                                                b, (const typename AccOf<P>::st*)yacc, scale, x, add_x, y))));
  return cudaGetLastError();
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st) { return cudaMemsetAsync(p, 0, bytes, st); }

}  // namespace ov
