// C-ABI entry points and host orchestration of the nested Krylov sign function.
//
// One call of ov_sign_apply runs, for a batch of right-hand sides sharing the gauge
// field and in lockstep:
//   pack x (norms -> v_1 = x/||x||)                        Sec. 2, Eq. (approximation)
//   for j = 1..: fused stencil step + vector update        Sec. 2 (Lanczos / two-sided Lanczos)
//     every check_interval steps: inner level on H_k       Sec. 3, Eqs. (nested), (precond)
//       (Roberts-Higham on the inner l x l matrix)         Sec. 2, Eq. (Roberts)
//       and the stopping estimates
//   recombination y = ||x|| V_k c from the stored basis, or by regenerating v_j from
//   the stored coefficients in a second pass (double pass, Sec. 4).
// The only device->host traffic inside the loop is the per-check readback. Runs of steps
// between checks replay captured CUDA graphs; a check runs on a second, high-priority
// stream while speculative steps continue (results as in the serial order); with learned
// sizing the first check goes to the predicted k*; with opts.relax the late steps use
// float hopping (both passes switch at the same step).
#include <math.h>
#include <stdio.h>

#include <cmath>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <climits>

#include <algorithm>
#include <complex>
#include <map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ov_internal.h"

using namespace ov;

// NVTX range around a phase (outer steps, a check, recombination), for timeline tools;
// costs a few nanoseconds when no tool is attached
struct Phase {
  explicit Phase(const char* name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
  Phase(const Phase&) = delete;
  Phase& operator=(const Phase&) = delete;
};

namespace {

constexpr int kChunk = 64;       // outer basis slots per allocation chunk
constexpr int kSizerSteps = 16;  // outer steps whose coefficients feed the learned sizing
constexpr int kSpecSteps = 24;   // speculative outer steps run while a check is evaluated
constexpr double kSpecFactor = 8.0;  // no speculation when the last estimate was within this of tol

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

cudaError_t grow(Buf& b, size_t bytes) {
  if (b.bytes >= bytes) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return e;
  }
  b.bytes = bytes;
  return cudaSuccess;
}
void release(Buf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

}  // namespace

struct TuneKey {
  int prec, mode, nprob, pad;
  bool operator<(const TuneKey& o) const {
    return prec != o.prec ? prec < o.prec : (mode != o.mode ? mode < o.mode : nprob < o.nprob);
  }
};

// one gauge field with its operator parameters
struct Lattice {
  Geometry g{};
  Buf links;
  double m_w = -1.5, mu = 0.0;
};

struct ov_handle {
  int dev = 0;
  cudaStream_t st = nullptr;
  int prec = OV_PREC_FP64;
  int antiperiodic = 1;
  ov_opts o{};
  // a single-field handle has one lattice and any number of right-hand sides per call;
  // a batch handle (ov_batch_create) has one lattice per problem and one source each
  std::vector<Lattice> lat;
  int is_batch = 0;
  Buf desc, blkmap;  // device problem descriptors and block -> problem map of the current call
  // outer level
  Buf xcanon, ycanon;             // canonical device copies for host buffers
  Buf tv, tw, p, r, vring, wring;  // [nrhs][12V] vectors (rings hold 2 slots)
  Buf yacc;                       // two-pass accumulator
  std::vector<Buf> chunks;        // stored basis: chunk c holds slots c*kChunk.. [slot][rhs][12V]
  size_t chunk_pool = 0;          // vector-pool bytes the chunks were sized for
  Buf coef_alp, coef_bet, coef_gam, coef_nv, coef_nw, coef_status, coef_kbreak;
  Buf partials, counters, scale, scal;
  int cap_rhs = 0, cap_ld = 0;
  // inner level
  Buf iQ, iT, ileff, iS, is, irh_its, irh_ok, iperm, ifail;
  Buf ck, cl, ckprev, cc_cur, cc_prev, cc_fin, cacc_cur, cacc_fin, c_est_in, c_est_out, c_rhst, c_rhit;
  Buf vptr;  // device array of basis slot pointers for recombination
  int inner_cap = 0, inner_ld = 0;
  ov_stats stats{};
  std::map<TuneKey, int> tuned;  // autotuned block size per (precision, mode, problem count)
  // CUDA graph of graph_steps outer steps (captured on a private stream, replayed on st)
  Buf jstate, slot_tab;
  cudaStream_t cap_st = nullptr;
  // stopping checks overlapped with speculative outer steps: a high-priority stream and
  // the events that order it against the handle's stream
  cudaStream_t chk_st = nullptr;
  cudaEvent_t ev_step = nullptr, ev_chk = nullptr;
  // captured graphs of U outer steps, one per step precision (strict and relaxed steps)
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    StepArgs args{};
    int U = 0, prec = -1, mode = -1;
  } graphs[2];
  // learned sizing
  Buf sizer_theta, sizer_feat, sizer_pred;
  int sizer_on = 0, sizer_lmin = 8, sizer_lmax = kMaxL;
  // the last apply (for ov_get_coefficients)
  int last_steps = 0, last_ld = 0, last_nrhs = 0;
  int trace = 0;  // OV_TRACE set in the environment: one JSON line per check on stderr
  size_t basis_cap = 0;  // OV_BASIS_CAP_BYTES: bytes the stored basis may take (0: no cap)
  Buf nn_scratch;        // the non-nested check's dense H_k, iterates and elimination buffers
  // deflation (Sec. 2): per lattice the critical eigenvalues and right / left eigenvectors
  // (canonical complex doubles, [m][12 V]; L = R at mu = 0)
  struct Defl {
    int m = 0;
    std::vector<std::complex<double>> lam;
    std::vector<double> res;
    Buf R, L;
  };
  std::vector<Defl> defl;
  Buf dx, dy, dpart, dG;  // the deflated apply's source, result and coefficient scratch
  // event pairs recorded around timed launches: (class, start, stop)
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_class;
  std::vector<cudaStream_t> ev_stream;
  size_t ev_used = 0;
};

enum { kClsStencil = 0, kClsUpdate = 1, kClsInner = 2, kClsRecomb = 3, kClsTotal = 4, kClsRelaxed = 5 };

// record the start event of a timed launch group (no-op unless opts.timing)
static int tstart(ov_handle* h, int cls, cudaStream_t s = nullptr) {
  if (!h->o.timing) return -1;
  if (h->ev_used + 2 > h->ev_pool.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      h->ev_pool.push_back(e);
    }
    h->ev_class.resize(h->ev_pool.size() / 2);
    h->ev_stream.resize(h->ev_pool.size() / 2);
  }
  const int slot = (int)(h->ev_used / 2);
  h->ev_class[slot] = cls;
  h->ev_stream[slot] = s ? s : h->st;
  cudaEventRecord(h->ev_pool[h->ev_used], h->ev_stream[slot]);
  h->ev_used += 2;
  return slot;
}
static void tstop(ov_handle* h, int slot) {
  if (slot < 0) return;
  cudaEventRecord(h->ev_pool[2 * slot + 1], h->ev_stream[slot]);
}
// after the stream has drained: add the recorded durations to the statistics
static void tcollect(ov_handle* h) {
  for (size_t s = 0; s < h->ev_used / 2; ++s) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[2 * s], h->ev_pool[2 * s + 1]) != cudaSuccess) continue;
    switch (h->ev_class[s]) {
      case kClsStencil: h->stats.stencil_ms += ms; break;
      case kClsRelaxed:
        h->stats.stencil_ms += ms;
        h->stats.relaxed_ms += ms;
        break;
      case kClsUpdate: h->stats.update_ms += ms; break;
      case kClsInner: h->stats.inner_ms += ms; break;
      case kClsRecomb: h->stats.recombine_ms += ms; break;
      default: h->stats.total_ms += ms; break;
    }
  }
  h->ev_used = 0;
}

extern "C" int ov_get_stats(const ov_handle* h, ov_stats* s) {
  if (!h || !s) return OV_ERR_ARG;
  *s = h->stats;
  return OV_OK;
}

extern "C" int ov_reset_stats(ov_handle* h) {
  if (!h) return OV_ERR_ARG;
  h->stats = ov_stats{};
  return OV_OK;
}

#define CK(call)                                       \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) {                           \
      fprintf(stderr, "libov: %s failed: %s (%s:%d)\n", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? OV_ERR_NOMEM : OV_ERR_CUDA; \
    }                                                  \
  } while (0)

// Problem descriptors of one call: problem r uses lattice lat_of[r]; vectors are pooled
// (12 V_r complex entries per problem, in problem order). Uploads the descriptors and the
// block map and returns the batch description and the pool size in complex entries.
// Site blocks in an order that keeps the neighbour planes of a block recently touched: the
// blocks are bs consecutive sites (x fastest), so the +-x (and mostly +-y) hops stay inside a
// block and the +-z, +-t hops reach other blocks; sorting the blocks by the Morton code of
// the (y, z, t) coordinates of their first site brings those blocks close in launch order,
// so their vectors are still in L2 when the neighbours read them. The reductions index their
// partial sums by the site block, so the order changes no result.
static std::vector<int> block_order(const Geometry& g, int bs) {
  const int nb = num_site_blocks(g, bs);
  std::vector<std::pair<unsigned long long, int>> key(nb);
  for (int q = 0; q < nb; ++q) {
    const long long s = (long long)q * bs;
    const unsigned y = (unsigned)((s / g.Lx) % g.Ly), z = (unsigned)((s / ((long long)g.Lx * g.Ly)) % g.Lz),
                   t = (unsigned)(s / ((long long)g.Lx * g.Ly * g.Lz));
    unsigned long long m = 0;
    for (int bit = 0; bit < 16; ++bit) {
      m |= (unsigned long long)((y >> bit) & 1u) << (3 * bit);
      m |= (unsigned long long)((z >> bit) & 1u) << (3 * bit + 1);
      m |= (unsigned long long)((t >> bit) & 1u) << (3 * bit + 2);
    }
    key[q] = {m, q};
  }
  std::sort(key.begin(), key.end());
  std::vector<int> ord(nb);
  for (int q = 0; q < nb; ++q) ord[q] = key[q].second;
  return ord;
}

static int build_batch(ov_handle* h, const std::vector<int>& lat_of, int bs, Batch* b, size_t* pool,
                       int neg_mu = 0) {
  const int np = (int)lat_of.size();
  std::vector<ProbDesc> d(np);
  std::vector<int2> map;
  size_t voff = 0;
  int blk = 0;
  bool same_lattice = true;
  for (int r = 0; r < np; ++r) {
    const Lattice& L = h->lat[lat_of[r]];
    d[r].g = L.g;
    d[r].links = L.links.p;
    fill_consts(d[r], L.m_w, neg_mu ? -L.mu : L.mu);
    d[r].voff = voff;
    d[r].block0 = blk;
    d[r].nblk = num_site_blocks(L.g, bs);
    voff += 12 * (size_t)L.g.V;
    blk += d[r].nblk;
    same_lattice = same_lattice && lat_of[r] == lat_of[0];
  }
  // Right-hand sides of one lattice: site-block-major order, so the blocks of every
  // right-hand side on the same sites run together and share the links (and neighbour
  // planes) in L2. Different lattices: problem-major.
  if (same_lattice) {
    for (int q : block_order(d[0].g, bs))
      for (int r = 0; r < np; ++r) map.push_back(make_int2(r, q));
  } else {
    for (int r = 0; r < np; ++r)
      for (int q : block_order(d[r].g, bs)) map.push_back(make_int2(r, q));
  }
  CK(grow(h->desc, sizeof(ProbDesc) * np));
  CK(grow(h->blkmap, sizeof(int2) * map.size()));
  CK(cudaMemcpyAsync(h->desc.p, d.data(), sizeof(ProbDesc) * np, cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->blkmap.p, map.data(), sizeof(int2) * map.size(), cudaMemcpyHostToDevice, h->st));
  b->desc = (const ProbDesc*)h->desc.p;
  b->blk_map = (const int2*)h->blkmap.p;
  b->nblocks = blk;
  b->nprob = np;
  b->block = bs;
  *pool = voff;
  return OV_OK;
}

// site blocks of a call at the smallest block size (sizes the partial-sum buffer)
static int max_blocks(const ov_handle* h, const std::vector<int>& lat_of) {
  int n = 0;
  for (int q : lat_of) n += num_site_blocks(h->lat[q].g, 64);
  return n;
}

static std::vector<int> lattices_of_call(const ov_handle* h, int nprob) {
  std::vector<int> v(nprob, 0);
  if (h->is_batch)
    for (int r = 0; r < nprob; ++r) v[r] = r;
  return v;
}

extern "C" void ov_default_opts(ov_opts* o) {
  if (!o) return;
  o->check_interval = 10;
  o->first_check = 0;
  o->recombination = OV_RECOMB_AUTO;
  o->rh_tol = 1e-10;
  o->rh_maxit = 100;
  o->breakdown_tol = 1e-14;
  o->inner_dl = 4;
  o->k_fixed = 0;
  o->check_schedule = 0;
  o->block_size = 0;
  o->graph_steps = 8;
  o->timing = 0;
  o->inner_arith = OV_INNER_DF64;
  o->relax = 0.0;
  o->overlap_checks = 1;
  o->nested = 1;
  o->rh_scaling = 1;
}

extern "C" const char* ov_strerror(int code) {
  switch (code) {
    case OV_OK: return "ok";
    case OV_NOT_CONVERGED: return "not converged (tolerance not reached at k_max or inner dimension too small)";
    case OV_ERR_ARG: return "invalid argument";
    case OV_ERR_NOMEM: return "device allocation failed";
    case OV_ERR_CUDA: return "CUDA error";
    case OV_ERR_BREAKDOWN: return "serious breakdown of the two-sided Lanczos recurrence";
    case OV_ERR_RH_NOCONV: return "Roberts-Higham iteration did not converge";
    case OV_ERR_TOO_LARGE: return "size exceeds a device limit";
    default: return "unknown status";
  }
}

static int check_opts(const ov_opts& o) {
  if (o.check_interval < 1 || o.rh_maxit < 1 || !(o.rh_tol > 0) || o.inner_dl < 1 || o.k_fixed < 0 ||
      o.first_check < 0 || o.recombination < 0 || o.recombination > 2 || !(o.breakdown_tol >= 0) ||
      o.check_schedule < 0 || o.check_schedule > 1 ||
      (o.block_size != 0 && o.block_size != 64 && o.block_size != 128 && o.block_size != 256) ||
      o.graph_steps < 0 || o.graph_steps > 256 || o.inner_arith < 0 || o.inner_arith > 1 ||
      !(o.relax >= 0.0 && o.relax <= 1.0) || o.overlap_checks < 0 || o.overlap_checks > 1 || o.nested < 0 ||
      o.nested > 1 || o.rh_scaling < 0 || o.rh_scaling > 1)
    return OV_ERR_ARG;
  return OV_OK;
}

extern "C" int ov_set_opts(ov_handle* h, const ov_opts* opts) {
  if (!h || !opts) return OV_ERR_ARG;
  if (check_opts(*opts) != OV_OK) return OV_ERR_ARG;
  h->o = *opts;
  return OV_OK;
}

// canonical links [V][4][3][3] -> [4][9][V], t-boundary sign folded into U_t(t = Lt-1)
template <class T>
__global__ void k_links(Geometry g, int anti, const double2* __restrict__ in, T* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const int t = s / (g.Lx * g.Ly * g.Lz);
  for (int nu = 0; nu < 4; ++nu) {
    const double sg = (nu == 3 && anti && t == g.Lt - 1) ? -1.0 : 1.0;
    for (int e = 0; e < 9; ++e) {
      const double2 z = in[((size_t)s * 4 + nu) * 9 + e];
      T o;
      o.x = sg * z.x;
      o.y = sg * z.y;
      out[(size_t)(nu * 9 + e) * g.V + s] = o;
    }
  }
}

// double-float links: the float pairs (hi, lo) with hi + lo = U to 2^-48 relative,
// stored as two planes [4][9][V] of float2 (hi first, then lo)
__global__ void k_links_df(Geometry g, int anti, const double2* __restrict__ in, float2* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const int t = s / (g.Lx * g.Ly * g.Lz);
  float2* lo = out + (size_t)36 * g.V;
  for (int nu = 0; nu < 4; ++nu) {
    const double sg = (nu == 3 && anti && t == g.Lt - 1) ? -1.0 : 1.0;
    for (int e = 0; e < 9; ++e) {
      const double2 z = in[((size_t)s * 4 + nu) * 9 + e];
      const double x = sg * z.x, y = sg * z.y;
      const float xh = (float)x, yh = (float)y;
      out[(size_t)(nu * 9 + e) * g.V + s] = make_float2(xh, yh);
      lo[(size_t)(nu * 9 + e) * g.V + s] = make_float2((float)(x - (double)xh), (float)(y - (double)yh));
    }
  }
}

extern "C" int ov_create(ov_handle** hp, const ov_geom* geom, const void* links, int links_mem, double m_w,
                         double mu, const ov_opts* opts, void* stream) {
  if (!hp || !geom || !links) return OV_ERR_ARG;
  *hp = nullptr;
  if (!(m_w > -2.0 && m_w < 0.0) || !isfinite(mu)) return OV_ERR_ARG;  // -2 < m_w < 0 (Sec. 1)
  for (int d = 0; d < 4; ++d)
    if (geom->dims[d] < 2) return OV_ERR_ARG;
  if (geom->precision < 0 || geom->precision > 2) return OV_ERR_ARG;
  if (links_mem != OV_MEM_HOST && links_mem != OV_MEM_DEVICE) return OV_ERR_ARG;
  const long long V = (long long)geom->dims[0] * geom->dims[1] * geom->dims[2] * geom->dims[3];
  if (V > (1LL << 30) / 12) return OV_ERR_TOO_LARGE;
  ov_opts o;
  ov_default_opts(&o);
  if (opts) {
    if (check_opts(*opts) != OV_OK) return OV_ERR_ARG;
    o = *opts;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return OV_ERR_CUDA;
  ov_handle* h = new ov_handle();
  CK(cudaGetDevice(&h->dev));
  h->st = (cudaStream_t)stream;
  h->lat.resize(1);
  Lattice& L = h->lat[0];
  L.g = Geometry{(int)V, geom->dims[0], geom->dims[1], geom->dims[2], geom->dims[3]};
  L.m_w = m_w;
  L.mu = mu;
  h->prec = geom->precision;
  h->antiperiodic = geom->t_antiperiodic ? 1 : 0;
  h->o = o;
  h->trace = getenv("OV_TRACE") != nullptr;
  if (const char* cap = getenv("OV_BASIS_CAP_BYTES")) h->basis_cap = (size_t)strtoull(cap, nullptr, 10);
  const size_t canon = sizeof(double2) * 36 * (size_t)V;
  const double2* src = (const double2*)links;
  Buf tmp;
  auto fail = [&](int code) {
    release(tmp);
    ov_destroy(h);
    return code;
  };
  if (links_mem == OV_MEM_HOST) {
    if (grow(tmp, canon) != cudaSuccess) return fail(OV_ERR_NOMEM);
    if (cudaMemcpyAsync(tmp.p, links, canon, cudaMemcpyHostToDevice, h->st) != cudaSuccess) return fail(OV_ERR_CUDA);
    src = (const double2*)tmp.p;
  }
  // FP64: double links; FP32: float links; DF64: float hi and lo planes
  const size_t lb = (h->prec == OV_PREC_FP32 ? 1 : 2) * sizeof(float2) * 36 * (size_t)V;
  if (grow(L.links, lb) != cudaSuccess) return fail(OV_ERR_NOMEM);
  const int nb = (int)((V + 127) / 128);
  if (h->prec == OV_PREC_FP64)
    k_links<double2><<<nb, 128, 0, h->st>>>(L.g, h->antiperiodic, src, (double2*)L.links.p);
  else if (h->prec == OV_PREC_DF64)
    k_links_df<<<nb, 128, 0, h->st>>>(L.g, h->antiperiodic, src, (float2*)L.links.p);
  else
    k_links<float2><<<nb, 128, 0, h->st>>>(L.g, h->antiperiodic, src, (float2*)L.links.p);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->st) != cudaSuccess) return fail(OV_ERR_CUDA);
  release(tmp);
  *hp = h;
  return OV_OK;
}

extern "C" void ov_destroy(ov_handle* h) {
  if (!h) return;
  cudaSetDevice(h->dev);
  if (h->st) cudaStreamSynchronize(h->st);
  for (Lattice& L : h->lat) release(L.links);
  Buf* all[] = {&h->desc, &h->blkmap, &h->xcanon, &h->ycanon, &h->tv, &h->tw, &h->p, &h->r, &h->vring, &h->wring, &h->yacc,
                &h->coef_alp, &h->coef_bet, &h->coef_gam, &h->coef_nv, &h->coef_nw, &h->coef_status,
                &h->coef_kbreak, &h->partials, &h->counters, &h->scale, &h->scal, &h->iQ, &h->iT, &h->ileff, &h->iS, &h->is,
                &h->irh_its, &h->irh_ok, &h->iperm, &h->ifail, &h->ck, &h->cl, &h->ckprev, &h->cc_cur, &h->cc_prev,
                &h->cc_fin, &h->cacc_cur, &h->cacc_fin, &h->c_est_in, &h->c_est_out, &h->c_rhst, &h->c_rhit,
                &h->vptr, &h->sizer_theta, &h->sizer_feat, &h->sizer_pred, &h->nn_scratch, &h->dx, &h->dy,
                &h->dpart, &h->dG};
  for (Buf* b : all) release(*b);
  for (Buf& b : h->chunks) release(b);
  for (auto& d : h->defl) {
    release(d.R);
    release(d.L);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  for (auto& gr : h->graphs)
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  if (h->chk_st) cudaStreamDestroy(h->chk_st);
  if (h->ev_step) cudaEventDestroy(h->ev_step);
  if (h->ev_chk) cudaEventDestroy(h->ev_chk);
  release(h->jstate);
  release(h->slot_tab);
  delete h;
}

// ---------------------------------------------------------------- workspace
static int ensure_outer(ov_handle* h, int nrhs, int ld, size_t pool, int nblocks) {
  const size_t vb = vec_elem_bytes(h->prec) * pool;
  CK(grow(h->tv, vb));
  CK(grow(h->tw, vb));
  CK(grow(h->p, vb));
  CK(grow(h->r, vb));
  CK(grow(h->vring, 2 * vb));
  CK(grow(h->wring, 2 * vb));
  const size_t cb = sizeof(double2) * (size_t)nrhs * ld;
  CK(grow(h->coef_alp, cb));
  CK(grow(h->coef_bet, cb));
  CK(grow(h->coef_gam, cb));
  CK(grow(h->coef_nw, cb));
  CK(grow(h->coef_nv, sizeof(double) * (size_t)nrhs * ld));
  CK(grow(h->coef_status, sizeof(int) * nrhs));
  CK(grow(h->coef_kbreak, sizeof(int) * nrhs));
  CK(grow(h->partials, sizeof(double) * 4 * (size_t)nblocks));
  if (h->counters.bytes < sizeof(unsigned) * nrhs) {
    CK(grow(h->counters, sizeof(unsigned) * nrhs));
    CK(cudaMemsetAsync(h->counters.p, 0, sizeof(unsigned) * nrhs, h->st));
  }
  CK(grow(h->scale, sizeof(double) * nrhs));
  CK(grow(h->scal, sizeof(float4) * 8 * (size_t)nrhs));
  h->cap_rhs = nrhs;
  h->cap_ld = ld;
  return OV_OK;
}

static int ensure_inner(ov_handle* h, int count, int ld) {
  // ld: leading dimension of the per-problem k-vectors (>= k + 2)
  CK(grow(h->iQ, sizeof(double2) * (size_t)count * ld * kMaxL));
  CK(grow(h->iT, sizeof(double2) * (size_t)count * kMaxL * 3));
  CK(grow(h->ileff, sizeof(int) * count));
  CK(grow(h->iS, sizeof(double2) * (size_t)2 * count * kMaxL * kMaxL));
  CK(grow(h->is, sizeof(double2) * (size_t)2 * count * kMaxL));
  CK(grow(h->irh_its, sizeof(int) * 2 * count));
  CK(grow(h->irh_ok, sizeof(int) * 2 * count));
  CK(grow(h->iperm, sizeof(int) * 2 * (size_t)count * kMaxL));
  CK(grow(h->ifail, sizeof(int) * count));
  const size_t cb = sizeof(double2) * (size_t)count * ld;
  CK(grow(h->ck, sizeof(int) * count));
  CK(grow(h->cl, sizeof(int) * count));
  CK(grow(h->ckprev, sizeof(int) * count));
  CK(grow(h->cc_cur, cb));
  CK(grow(h->cc_prev, cb));
  CK(grow(h->cc_fin, cb));
  const size_t ab = acc_elem_bytes(h->prec) * (size_t)count * ld;
  CK(grow(h->cacc_cur, ab));
  CK(grow(h->cacc_fin, ab));
  CK(grow(h->c_est_in, sizeof(double) * count));
  CK(grow(h->c_est_out, sizeof(double) * count));
  CK(grow(h->c_rhst, sizeof(int) * count));
  CK(grow(h->c_rhit, sizeof(int) * count));
  h->inner_cap = count;
  h->inner_ld = ld;
  return OV_OK;
}

static InnerWork inner_work(ov_handle* h) {
  InnerWork w;
  w.Q = (double2*)h->iQ.p;
  w.T = (double2*)h->iT.p;
  w.leff = (int*)h->ileff.p;
  w.S = (double2*)h->iS.p;
  w.s = (double2*)h->is.p;
  w.rh_its = (int*)h->irh_its.p;
  w.rh_ok = (int*)h->irh_ok.p;
  w.perm = (int*)h->iperm.p;
  w.fail = (int*)h->ifail.p;
  w.ld = h->inner_ld;  // Q rows per problem, as allocated by ensure_inner
  w.arith = h->o.inner_arith;
  w.rh_scale = h->o.rh_scaling;
  return w;
}

static Coefs coefs(ov_handle* h, int ld) {
  Coefs c;
  c.alp = (double2*)h->coef_alp.p;
  c.bet = (double2*)h->coef_bet.p;
  c.gam = (double2*)h->coef_gam.p;
  c.nv = (double*)h->coef_nv.p;
  c.nw = (double2*)h->coef_nw.p;
  c.status = (int*)h->coef_status.p;
  c.kbreak = (int*)h->coef_kbreak.p;
  c.ld = ld;
  return c;
}

// pointer to basis slot `slot` (0-based, = step j - 1), allocating chunks on demand
static int basis_slot(ov_handle* h, size_t pool_bytes, int slot, void** out) {
  if (h->chunk_pool != pool_bytes) {
    for (Buf& b : h->chunks) release(b);
    h->chunks.clear();
    h->chunk_pool = pool_bytes;
  }
  const int c = slot / kChunk;
  while ((int)h->chunks.size() <= c) {
    // a cap on the stored basis set from the environment (OV_BASIS_CAP_BYTES) behaves like
    // device memory running out at that point: how the fall-back to the double pass is tested
    if (h->basis_cap > 0 && pool_bytes * kChunk * (h->chunks.size() + 1) > h->basis_cap) return OV_ERR_NOMEM;
    Buf b;
    cudaError_t e = grow(b, pool_bytes * kChunk);
    if (e != cudaSuccess) {
      cudaGetLastError();  // clear the allocation error
      return OV_ERR_NOMEM;
    }
    h->chunks.push_back(b);
  }
  *out = (char*)h->chunks[c].p + pool_bytes * (size_t)(slot % kChunk);
  return OV_OK;
}

// A graph of U outer steps for these step arguments: captured once (on a private stream;
// the kernels take j and their slots from the device step state, so every replay runs
// the next U steps) and kept while the arguments stay the same.
static int graph_for(ov_handle* h, const StepArgs& a, int prec, int mode, int U, cudaGraphExec_t* out) {
  auto& gr = h->graphs[prec == kPrecDF64Relaxed ? 1 : 0];
  *out = nullptr;
  if (gr.exec && gr.U == U && gr.prec == prec && gr.mode == mode && memcmp(&gr.args, &a, sizeof(a)) == 0) {
    *out = gr.exec;
    return OV_OK;
  }
  if (gr.exec) {
    cudaGraphExecDestroy(gr.exec);
    gr.exec = nullptr;
  }
  if (!h->cap_st) CK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int u = 0; u < U && e == cudaSuccess; ++u) {
    e = launch_step(prec, mode, a, h->cap_st);
    if (e == cudaSuccess) e = launch_update(h->prec, mode, a, h->cap_st);
  }
  cudaError_t e2 = cudaStreamEndCapture(h->cap_st, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return OV_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&gr.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    gr.exec = nullptr;
    cudaGetLastError();
    return OV_ERR_CUDA;
  }
  gr.args = a;
  gr.U = U;
  gr.prec = prec;
  gr.mode = mode;
  *out = gr.exec;
  return OV_OK;
}

// ---------------------------------------------------------------- sign apply
static int sign_apply_core(ov_handle* h, int nrhs, const void* x, void* y, int mem, double tol, int k_max, int l,
                           ov_info* info, int add_x, int neg_mu = 0, int strict_only = 0) {
  const Phase ph_apply("ov_sign_apply");
  if (!h || !x || !y || nrhs < 1 || k_max < 1 || l < 1 || !(tol >= 0.0)) return OV_ERR_ARG;
  if (mem != OV_MEM_HOST && mem != OV_MEM_DEVICE) return OV_ERR_ARG;
  if (l > kMaxL) return OV_ERR_TOO_LARGE;
  const ov_opts& o = h->o;
  const int ktarget = o.k_fixed > 0 ? o.k_fixed : k_max;
  if (ktarget > kMaxInnerK) return OV_ERR_TOO_LARGE;
  CK(cudaSetDevice(h->dev));
  cudaStream_t st = h->st;
  if (h->is_batch && nrhs != (int)h->lat.size()) return OV_ERR_ARG;
  const std::vector<int> lat_of = lattices_of_call(h, nrhs);
  bool herm = true;
  for (int q : lat_of) herm = herm && h->lat[q].mu == 0.0;
  const int mode = herm ? kModeLanczos : kModeTwoSided;
  const int ld = ktarget + 2;
  Batch bt;
  size_t pool = 0;
  // block size: forced by opts.block_size, else the tuned one for this problem set, else
  // tuned below at the first step
  const TuneKey key{h->prec, mode, nrhs, 0};
  int bs = o.block_size;
  bool tune = false;
  if (bs == 0) {
    auto it = h->tuned.find(key);
    if (it != h->tuned.end()) bs = it->second;
    else { bs = kBlockDefault; tune = true; }
  }
  int rc = build_batch(h, lat_of, bs, &bt, &pool, neg_mu);
  if (rc != OV_OK) return rc;
  rc = ensure_outer(h, nrhs, ld, pool, max_blocks(h, lat_of));
  if (rc != OV_OK) return rc;
  rc = ensure_inner(h, nrhs, ld);
  if (rc != OV_OK) return rc;
  const size_t canon = sizeof(double2) * pool;
  const double2* xd = (const double2*)x;
  double2* yd = (double2*)y;
  if (mem == OV_MEM_HOST) {
    CK(grow(h->xcanon, canon));
    CK(grow(h->ycanon, canon));
    CK(cudaMemcpyAsync(h->xcanon.p, x, canon, cudaMemcpyHostToDevice, st));
    xd = (const double2*)h->xcanon.p;
    yd = (double2*)h->ycanon.p;
  }
  Coefs c = coefs(h, ld);
  const size_t vbn = vec_elem_bytes(h->prec) * pool;  // one vector of every problem
  CK(cudaMemsetAsync(c.alp, 0, sizeof(double2) * (size_t)nrhs * ld, st));
  CK(cudaMemsetAsync(c.bet, 0, sizeof(double2) * (size_t)nrhs * ld, st));
  CK(cudaMemsetAsync(c.gam, 0, sizeof(double2) * (size_t)nrhs * ld, st));
  CK(cudaMemsetAsync(h->vring.p, 0, 2 * vbn, st));
  CK(cudaMemsetAsync(h->wring.p, 0, 2 * vbn, st));
  // v_1 = w_1 = x / ||x||: x goes to tv (and tw), the norm into nv_1 / nw_1
  int recomb = o.recombination;
  if (recomb == OV_RECOMB_AUTO) {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    const size_t need = vbn * (size_t)(ktarget + 1);
    recomb = need + ((size_t)2 << 30) < fr ? OV_RECOMB_STORED : OV_RECOMB_TWO_PASS;
  }
  // t_1 = x (unnormalised, nv_1 = ||x||) goes to basis slot 0 (stored mode) or ring slot 1;
  // tw_1 = x to the w ring's slot 1; the zeroed ring slots 0 are t_0 = tw_0 = 0
  std::vector<void*> slots;  // device pointer of each stored t_j (stored mode): slots[i] = t_{i+1}
  if (recomb == OV_RECOMB_STORED) {
    void* s0 = nullptr;
    rc = basis_slot(h, vbn, 0, &s0);
    if (rc == OV_OK) slots.push_back(s0);
    else if (o.recombination == OV_RECOMB_AUTO) recomb = OV_RECOMB_TWO_PASS;
    else return rc;
  }
  void* t1 = recomb == OV_RECOMB_STORED ? slots[0] : (char*)h->vring.p + vbn;
  CK(launch_pack(h->prec, bt, xd, t1, herm ? nullptr : (char*)h->wring.p + vbn, c, (double*)h->partials.p,
                 (unsigned*)h->counters.p, 1, h->scal.p, st));
  CK(cudaMemcpy2DAsync(h->scale.p, sizeof(double), (double*)c.nv + 1, sizeof(double) * ld, sizeof(double), nrhs,
                       cudaMemcpyDeviceToDevice, st));
  h->stats.launches += 1;
  h->stats.other_launches += 1;
  const int t_total = tstart(h, kClsTotal);

  StepArgs a{};
  a.b = bt;
  a.scal = h->scal.p;
  a.p = h->p.p;
  a.r = h->r.p;
  a.c = c;
  a.breakdown_tol = o.breakdown_tol;
  a.partials = (double*)h->partials.p;
  a.counters = (unsigned*)h->counters.p;

  // host-side per-RHS state
  std::vector<int> done(nrhs, 0), kfin(nrhs, 0), lfin(nrhs, 0), itfin(nrhs, 0), stat(nrhs, OV_OK);
  std::vector<int> kprev(nrhs, 0), kcur(nrhs, 0), lreq(nrhs, std::min(l, kMaxL));
  std::vector<double> estfin(nrhs, INFINITY), estin(nrhs, NAN);
  std::vector<int> dstatus(nrhs), dkbreak(nrhs), rhst(nrhs), rhit(nrhs), leff(nrhs);
  std::vector<double> eo(nrhs), ei(nrhs);
  CK(cudaMemcpyAsync(h->cl.p, lreq.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(h->cc_fin.p, 0, sizeof(double2) * (size_t)nrhs * ld, st));
  CK(cudaMemsetAsync(h->cacc_fin.p, 0, acc_elem_bytes(h->prec) * (size_t)nrhs * ld, st));
  InnerWork iw = inner_work(h);
  int ndone = 0;
  int j = 0;
  const int first = o.first_check > 0 ? o.first_check : o.check_interval;
  int next_check = first;
  // last two (k, outer estimate) pairs per RHS for the adaptive schedule
  std::vector<double> hk1(nrhs, 0), he1(nrhs, 0), hk2(nrhs, 0), he2(nrhs, 0);
  std::vector<int> kprev_old(nrhs, 0);
  int last_check = 0;
  double eo_last_max = -1.0;  // largest outer estimate of the running RHS at the last check
  // device-side step state: j and the global ticket; the basis slot table; the rings
  {
    const int init[2] = {1, 0};
    CK(grow(h->jstate, sizeof(int) * 2));
    CK(cudaMemcpyAsync(h->jstate.p, init, sizeof(int) * 2, cudaMemcpyHostToDevice, st));
    CK(grow(h->slot_tab, sizeof(void*) * (size_t)(ktarget + 2)));
  }
  a.jdev = (int*)h->jstate.p;
  a.gticket = (unsigned*)((int*)h->jstate.p + 1);
  a.vring = h->vring.p;
  a.wring = h->wring.p;
  a.pool_bytes = vbn;
  a.slot_tab = recomb == OV_RECOMB_STORED ? (void* const*)h->slot_tab.p : nullptr;
  const int gU = (o.timing || o.graph_steps <= 0) ? 0 : o.graph_steps;
  // relaxed steps (double-float handles): float hopping from step relax_from on, the
  // same step in both passes; never on a deflated source (strict_only): the float
  // hopping error, ~1e-7 of |A v| in every direction, puts back components along the
  // removed eigenvectors, whose eigenvalues lie inside the deflation gap that the
  // shortened Krylov space no longer resolves
  const bool relaxing = !strict_only && o.relax > 0.0 && h->prec == OV_PREC_DF64;
  int relax_from = INT_MAX;
  if (relaxing) {
    if (o.k_fixed > 0) relax_from = std::max(1, (int)std::ceil(o.relax * o.k_fixed));
    else if (!h->sizer_on && o.first_check > 0) relax_from = std::max(1, (int)std::ceil(o.relax * o.first_check));
  }
  auto step_prec = [&](int jj) { return jj >= relax_from ? kPrecDF64Relaxed : h->prec; };
  int jdone = 0;
  size_t slots_on_device = 0;  // entries of the device slot table written so far
  // outer steps jfrom+1 .. jto: basis slots (stored mode), the autotuned block size at
  // step 1, whole graph units replayed and the rest launched one by one
  auto run_span = [&](int jfrom, int jto) -> int {
      const Phase ph_steps("outer steps");
      // basis slots of the span (stored mode), uploaded to the device slot table
      if (recomb == OV_RECOMB_STORED) {
        // slots up to index jto: the update of step jto writes t_{jto+1} there
        const size_t first_new = slots.size();
        const size_t upload_from = std::min(first_new, slots_on_device);
        for (int i = (int)slots.size(); i <= jto; ++i) {
          void* vc = nullptr;
          rc = basis_slot(h, vbn, i, &vc);
          if (rc != OV_OK) {
            if (o.recombination != OV_RECOMB_AUTO) return rc;
            // out of memory: fall back to the double pass from step jfrom + 1 on; the ring
            // gets t_{jfrom+1} and t_{jfrom} (t_0 = 0 is already in ring slot 0)
            recomb = OV_RECOMB_TWO_PASS;
            a.slot_tab = nullptr;
            CK(cudaMemcpyAsync((char*)h->vring.p + vbn * ((jfrom + 1) & 1), slots[jfrom], vbn,
                               cudaMemcpyDeviceToDevice, st));
            if (jfrom >= 1)
              CK(cudaMemcpyAsync((char*)h->vring.p + vbn * (jfrom & 1), slots[jfrom - 1], vbn,
                                 cudaMemcpyDeviceToDevice, st));
            slots.resize(first_new);
            break;
          }
          slots.push_back(vc);
        }
        if (recomb == OV_RECOMB_STORED && slots.size() > upload_from) {
          CK(cudaMemcpyAsync((void**)h->slot_tab.p + upload_from, slots.data() + upload_from,
                             sizeof(void*) * (slots.size() - upload_from), cudaMemcpyHostToDevice, st));
          slots_on_device = slots.size();
        }
      }
      int jn = jfrom + 1;
      if (jn == 1 && tune) {
        // autotune the block size on the first step (it only reads x and the step-1
        // scalars, so re-running it is harmless): best of two timed launches per size
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        float best = 1e30f;
        int best_bs = kBlockDefault;
        for (int cand : {64, 128, 256}) {
          Batch bc;
          size_t pc = 0;
          rc = build_batch(h, lat_of, cand, &bc, &pc, neg_mu);
          if (rc != OV_OK) return rc;
          a.b = bc;
          float tmin = 1e30f;
          for (int rep = 0; rep < 2; ++rep) {
            CK(cudaEventRecord(e0, st));
            CK(launch_step(h->prec, mode, a, st));
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            tmin = std::min(tmin, ms);
          }
          h->stats.launches += 2;
          if (tmin < best) { best = tmin; best_bs = cand; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        h->tuned[key] = best_bs;
        rc = build_batch(h, lat_of, best_bs, &bt, &pool, neg_mu);
        if (rc != OV_OK) return rc;
        a.b = bt;
        if (h->trace) fprintf(stderr, "{\"ov_autotune\": %d, \"ms\": %.4f}\n", best_bs, best);
      }
      h->stats.block_size = a.b.block;
      // steps jn..jto: whole graph units replayed, the rest launched one by one
      while (jn <= jto) {
        const int sp = step_prec(jn);
        // a graph unit holds steps of one precision
        if (gU > 0 && jto - jn + 1 >= gU && step_prec(jn + gU - 1) == sp) {
          cudaGraphExec_t gx = nullptr;
          rc = graph_for(h, a, sp, mode, gU, &gx);
          if (rc == OV_OK && gx) {
            CK(cudaGraphLaunch(gx, st));
            h->stats.launches += 2 * gU;
            h->stats.stencil_launches += gU;
            h->stats.update_launches += gU;
            h->stats.outer_steps += gU;
            h->stats.graph_launches += 1;
            if (sp == kPrecDF64Relaxed) h->stats.relaxed_steps += gU;
            jn += gU;
            continue;
          }
        }
        if (sp == kPrecDF64Relaxed) h->stats.relaxed_steps += 1;
        int ts = tstart(h, sp == kPrecDF64Relaxed ? kClsRelaxed : kClsStencil);
        CK(launch_step(sp, mode, a, st));
        tstop(h, ts);
        ts = tstart(h, kClsUpdate);
        CK(launch_update(h->prec, mode, a, st));
        tstop(h, ts);
        h->stats.launches += 2;
        h->stats.stencil_launches += 1;
        h->stats.update_launches += 1;
        h->stats.outer_steps += 1;
        ++jn;
      }
    return OV_OK;
  };
  // j: the step the loop has reached (the last check's, or the end of the last span);
  // jdone >= j: steps run so far, speculative steps run during a check included. The loop
  // ends when every right-hand side is done or the step at ktarget has been checked, also
  // where speculative steps already reached ktarget (then no step is run, only the check).
  for (;;) {
    if (j >= ktarget || ndone >= nrhs) break;
    const bool fixed_span = o.k_fixed > 0;
    int target = fixed_span ? ktarget : std::min(next_check, ktarget);
    if (h->sizer_on && !fixed_span && j < kSizerSteps && ktarget > kSizerSteps + 1)
      target = std::min(target, kSizerSteps);
    if (target <= j) target = j + 1;
    if (target > jdone) {
      rc = run_span(jdone, target);
      if (rc != OV_OK) return rc;
      jdone = target;
    }
    j = target;
    const bool fixed = o.k_fixed > 0;
    if (h->sizer_on && !fixed && j == kSizerSteps && ktarget > kSizerSteps + 1) {
      // learned sizing: f = (Re alpha_1..6, Im alpha_1..6, beta_2..5) -> (log k*, log l*)
      std::vector<double2> fa((size_t)nrhs * 6), fb((size_t)nrhs * 4);
      CK(cudaMemcpy2DAsync(fa.data(), sizeof(double2) * 6, c.alp + 1, sizeof(double2) * ld, sizeof(double2) * 6, nrhs,
                           cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpy2DAsync(fb.data(), sizeof(double2) * 4, c.bet + 2, sizeof(double2) * ld, sizeof(double2) * 4, nrhs,
                           cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      std::vector<float> feat((size_t)nrhs * 16), pred((size_t)nrhs * 2);
      for (int r = 0; r < nrhs; ++r) {
        for (int i = 0; i < 6; ++i) {
          feat[(size_t)r * 16 + i] = (float)fa[(size_t)r * 6 + i].x;
          feat[(size_t)r * 16 + 6 + i] = (float)fa[(size_t)r * 6 + i].y;
        }
        for (int i = 0; i < 4; ++i) feat[(size_t)r * 16 + 12 + i] = (float)fb[(size_t)r * 4 + i].x;
      }
      CK(grow(h->sizer_feat, sizeof(float) * feat.size()));
      CK(grow(h->sizer_pred, sizeof(float) * pred.size()));
      CK(cudaMemcpyAsync(h->sizer_feat.p, feat.data(), sizeof(float) * feat.size(), cudaMemcpyHostToDevice, st));
      CK(mlp_predict_device((const float*)h->sizer_theta.p, nrhs, (const float*)h->sizer_feat.p,
                            (float*)h->sizer_pred.p, st));
      CK(cudaMemcpyAsync(pred.data(), h->sizer_pred.p, sizeof(float) * pred.size(), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      h->stats.launches += 1;
      // the right-hand sides advance together until the last one stops, so the first
      // check goes to the largest predicted k*
      double kmax_pred = -1.0;
      for (int r = 0; r < nrhs; ++r) {
        const double kp = std::exp((double)pred[(size_t)r * 2]);
        const double lp = std::exp((double)pred[(size_t)r * 2 + 1]);
        if (std::isfinite(kp)) kmax_pred = std::max(kmax_pred, kp);
        int lr = std::isfinite(lp) ? ((int)std::ceil(lp / 8.0)) * 8 : h->sizer_lmax;
        lreq[r] = std::max(h->sizer_lmin, std::min(lr, std::min(h->sizer_lmax, std::min(l, kMaxL))));
      }
      CK(cudaMemcpyAsync(h->cl.p, lreq.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
      // (at most one interval before k_max, so that the check at k_max has a baseline)
      if (kmax_pred > 0.0)
        next_check = std::max(j + 1, std::min((int)std::floor(std::min(kmax_pred, (double)ktarget)),
                                              ktarget - o.check_interval));
      if (relaxing && kmax_pred > 0.0)
        relax_from = std::max(j + 1, (int)std::ceil(o.relax * std::min(kmax_pred, (double)ktarget)));
      if (h->trace)
        fprintf(stderr, "{\"ov_sizer\": %d, \"k_pred_max\": %.1f, \"l_req0\": %d, \"relax_from\": %d}\n", j,
                kmax_pred, lreq[0], relaxing ? relax_from : -1);
    }
    const bool check = fixed ? (j == ktarget) : (j >= next_check || j == ktarget);
    if (!check) continue;
    // the check runs on the check stream while speculative outer steps (at most
    // kSpecSteps, never past the next check) run on the handle's stream; they only add
    // coefficients and basis vectors beyond k = j, so the check and the result are those of
    // the serial order, and the steps count towards the next interval if the run goes on
    cudaStream_t cs = st;
    int spec = 0;
    // (not before the learned sizing has read its 16 steps: it runs where a span ends there;
    // and not where the run is likely to stop: the previous check's largest outer estimate
    // within kSpecFactor of tol. The choice only moves time, never the result)
    const bool likely_stop = eo_last_max >= 0.0 && eo_last_max <= kSpecFactor * tol;
    if (o.overlap_checks && !fixed && j < ktarget && !(h->sizer_on && j < kSizerSteps) && !likely_stop) {
      spec = std::min(std::min(kSpecSteps, o.check_interval - 1), ktarget - j);
      if (spec > 0) {
        if (!h->chk_st) {
          int lo = 0, hi = 0;
          CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
          CK(cudaStreamCreateWithPriority(&h->chk_st, cudaStreamNonBlocking, hi));
          CK(cudaEventCreateWithFlags(&h->ev_step, cudaEventDisableTiming));
          CK(cudaEventCreateWithFlags(&h->ev_chk, cudaEventDisableTiming));
        }
        CK(cudaEventRecord(h->ev_step, st));
        rc = run_span(j, j + spec);
        if (rc != OV_OK) return rc;
        CK(cudaStreamWaitEvent(h->chk_st, h->ev_step, 0));
        cs = h->chk_st;
      }
    }
    // read the breakdown state first: a Lanczos breakdown fixes k for that RHS
    CK(cudaMemcpyAsync(dstatus.data(), c.status, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, cs));
    CK(cudaMemcpyAsync(dkbreak.data(), c.kbreak, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, cs));
    CK(cudaStreamSynchronize(cs));
    // a breakdown recorded by a speculative step (after j) is not part of this check; one at
    // or before j has both words written before the check began (a pair still being written
    // by a running speculative step can show the status without its step)
    for (int r = 0; r < nrhs; ++r)
      if ((dstatus[r] == kStLucky || dstatus[r] == kStBreakdown) && (dkbreak[r] <= 0 || dkbreak[r] > j))
        dstatus[r] = kStOK;
    for (int r = 0; r < nrhs; ++r) kcur[r] = (dstatus[r] != kStOK && dkbreak[r] > 0) ? std::min(dkbreak[r], j) : j;
    CK(cudaMemcpyAsync(h->ck.p, kcur.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, cs));
    CK(cudaMemcpyAsync(h->ckprev.p, kprev.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, cs));
    const Phase ph_check("stopping check");
    bool regrow = false;
    do {
    regrow = false;
    const auto tc0 = std::chrono::steady_clock::now();
    const int ti = tstart(h, kClsInner, cs);
    // where a stop is likely, both Roberts-Higham sets (the inner estimate's too) in one
    // launch instead of a second round trip
    // (the non-nested check has no inner estimate to defer)
    const int phase = (!o.nested || (likely_stop && !fixed)) ? 0 : 1;
    cudaError_t e;
    if (!o.nested) {
      CK(grow(h->nn_scratch, nonnested_scratch_bytes(nrhs, *std::max_element(kcur.begin(), kcur.end()))));
      e = run_nonnested(nrhs, kcur.data(), c.alp, c.bet, c.gam, c.nv, ld, o.rh_tol, o.rh_maxit, (double2*)h->cc_cur.p,
                        ld, h->cacc_cur.p, h->prec, (double*)h->c_est_in.p, (const double2*)h->cc_prev.p, ld,
                        (const int*)h->ckprev.p, (double*)h->c_est_out.p, (int*)h->c_rhst.p, (int*)h->c_rhit.p,
                        h->nn_scratch.p, cs);
    } else
    e = run_inner(nrhs, (const int*)h->ck.p, (const int*)h->cl.p, herm ? 1 : 0, c.alp, c.bet, c.gam, c.nv, ld, iw,
                              o.rh_tol, o.rh_maxit, o.inner_dl, (double2*)h->cc_cur.p, ld, h->cacc_cur.p, h->prec,
                              (double*)h->c_est_in.p, (const double2*)h->cc_prev.p, ld, (const int*)h->ckprev.p,
                              (double*)h->c_est_out.p, (int*)h->c_rhst.p, (int*)h->c_rhit.p, phase, cs);
    CK(e);
    tstop(h, ti);
    h->stats.launches += 3;
    h->stats.inner_launches += 3;
    h->stats.checks += 1;
    CK(cudaMemcpyAsync(eo.data(), h->c_est_out.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, cs));
    CK(cudaMemcpyAsync(rhst.data(), h->c_rhst.p, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, cs));
    CK(cudaMemcpyAsync(rhit.data(), h->c_rhit.p, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, cs));
    CK(cudaMemcpyAsync(leff.data(), h->ileff.p, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, cs));
    CK(cudaStreamSynchronize(cs));
    // the inner estimate is needed only where the run may stop at this check
    bool want_inner = false;
    for (int r = 0; r < nrhs && !fixed; ++r)
      if (!done[r] && dstatus[r] != kStZero && dstatus[r] != kStBreakdown && rhst[r] == 0 &&
          (eo[r] <= tol || dstatus[r] == kStLucky || j == ktarget))
        want_inner = true;
    std::fill(ei.begin(), ei.end(), NAN);
    if (want_inner && phase == 0) {
      CK(cudaMemcpyAsync(ei.data(), h->c_est_in.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, cs));
      CK(cudaStreamSynchronize(cs));
    } else if (want_inner) {
      const int t2 = tstart(h, kClsInner, cs);
      e = run_inner(nrhs, (const int*)h->ck.p, (const int*)h->cl.p, herm ? 1 : 0, c.alp, c.bet, c.gam, c.nv, ld, iw, o.rh_tol,
                    o.rh_maxit, o.inner_dl, (double2*)h->cc_cur.p, ld, h->cacc_cur.p, h->prec,
                    (double*)h->c_est_in.p, (const double2*)h->cc_prev.p, ld, (const int*)h->ckprev.p,
                    (double*)h->c_est_out.p, (int*)h->c_rhst.p, (int*)h->c_rhit.p, 2, cs);
      CK(e);
      tstop(h, t2);
      h->stats.launches += 2;
      h->stats.inner_launches += 2;
      CK(cudaMemcpyAsync(ei.data(), h->c_est_in.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, cs));
      CK(cudaMemcpyAsync(rhst.data(), h->c_rhst.p, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, cs));
      CK(cudaStreamSynchronize(cs));
    }
    if (h->trace) {
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tc0).count();
      fprintf(stderr, "{\"ov_check\": %d, \"ms\": %.3f, \"speculative_steps\": %d, \"inner_estimate\": %d, \"rh_iters\": [",
              j, ms, spec, want_inner ? 1 : 0);
      for (int r = 0; r < nrhs; ++r) fprintf(stderr, "%s%d", r ? "," : "", rhit[r]);
      fprintf(stderr, "], \"est_outer\": [");
      for (int r = 0; r < nrhs; ++r) fprintf(stderr, "%s%.3e", r ? "," : "", eo[r]);
      fprintf(stderr, "], \"l_eff\": [");
      for (int r = 0; r < nrhs; ++r) fprintf(stderr, "%s%d", r ? "," : "", leff[r]);
      fprintf(stderr, "]}\n");
    }
    kprev_old = kprev;
    for (int r = 0; r < nrhs; ++r) {
      if (done[r]) continue;
      int fin = 0, sr = OV_OK;
      double est = eo[r];
      const bool lucky = dstatus[r] == kStLucky;
      const bool broke = dstatus[r] == kStBreakdown;
      if (dstatus[r] == kStZero) {
        // zero source: y = 0 exactly, nothing to iterate
        done[r] = 1;
        ++ndone;
        kfin[r] = 0;
        estfin[r] = 0.0;
        estin[r] = 0.0;
        stat[r] = OV_OK;
        continue;
      }
      if (rhst[r] != 0) {
        fin = 1;
        sr = OV_ERR_RH_NOCONV;
      } else if (broke) {
        fin = 1;
        sr = OV_ERR_BREAKDOWN;
      } else if (fixed) {
        fin = 1;
        est = NAN;
      } else {
        if (lucky) est = 0.0;
        if (est <= tol || lucky || j == ktarget) {
          // with learned sizing, an inner estimate above tol grows l and re-checks
          if (h->sizer_on && ei[r] > tol && lreq[r] < std::min(h->sizer_lmax, std::min(kcur[r], kMaxL))) {
            lreq[r] = std::min(lreq[r] + 16, std::min(h->sizer_lmax, kMaxL));
            regrow = true;
            continue;
          }
          fin = 1;
          est = std::max(est, ei[r]);
          sr = est <= tol ? OV_OK : OV_NOT_CONVERGED;
        }
      }
      if (fin) {
        done[r] = 1;
        ++ndone;
        kfin[r] = kcur[r];
        lfin[r] = leff[r];
        itfin[r] = rhit[r];
        estfin[r] = est;
        estin[r] = ei[r];
        stat[r] = sr;
        CK(cudaMemcpyAsync((double2*)h->cc_fin.p + (size_t)r * ld, (double2*)h->cc_cur.p + (size_t)r * ld,
                           sizeof(double2) * ld, cudaMemcpyDeviceToDevice, cs));
        const size_t ab = acc_elem_bytes(h->prec);
        CK(cudaMemcpyAsync((char*)h->cacc_fin.p + ab * (size_t)r * ld, (char*)h->cacc_cur.p + ab * (size_t)r * ld,
                           ab * ld, cudaMemcpyDeviceToDevice, cs));
      } else {
        kprev[r] = kcur[r];
        // est_outer compares with the previous check, so it measures the error there;
        // keep the first and the latest such point (the longest baseline for the rate,
        // since the decay is irregular over short spans)
        if (std::isfinite(eo[r]) && eo[r] > 0.0) {
          if (he1[r] <= 0.0) {
            hk1[r] = kprev_old[r];
            he1[r] = eo[r];
          } else {
            hk2[r] = kprev_old[r];
            he2[r] = eo[r];
          }
        }
      }
    }
    if (regrow) CK(cudaMemcpyAsync(h->cl.p, lreq.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, cs));
    } while (regrow);
    eo_last_max = 0.0;  // an estimate without a previous check (infinite) means unknown
    for (int r = 0; r < nrhs; ++r)
      if (!done[r]) eo_last_max = std::max(eo_last_max, std::isnan(eo[r]) ? INFINITY : eo[r]);
    if (cs != st) {
      // later work on the handle's stream (the final combination) reads the check's results
      CK(cudaEventRecord(h->ev_chk, cs));
      CK(cudaStreamWaitEvent(st, h->ev_chk, 0));
      jdone = j + spec;
    }
    std::swap(h->cc_cur, h->cc_prev);
    // next check: fixed interval, or (adaptive) a jump to where the log-linear decay of
    // the error reaches tol, always followed by a partner check check_interval later
    // (the estimate at a check measures the error at the check before it)
    int step = o.check_interval;
    if (o.check_schedule == 1 && j - last_check <= o.check_interval) {
      int pred = -1;
      for (int r = 0; r < nrhs; ++r) {
        if (done[r] || he1[r] <= 0.0 || he2[r] <= 0.0 || he2[r] >= he1[r] || tol <= 0.0 || hk2[r] <= hk1[r]) continue;
        const double rate = (std::log(he2[r]) - std::log(he1[r])) / (hk2[r] - hk1[r]);
        const double ks = hk2[r] + (std::log(tol) - std::log(he2[r])) / rate;
        // the batch runs until its slowest right-hand side stops: aim at the largest k*
        const int ahead = (int)std::ceil(ks) - j;
        if (ahead > pred) pred = ahead;
      }
      if (pred > step) step = std::min(pred, 4 * o.check_interval);
    }
    last_check = j;
    next_check = j + step;
  }
  const int kmax_used = *std::max_element(kfin.begin(), kfin.end());
  h->last_steps = jdone;
  h->last_ld = ld;
  h->last_nrhs = nrhs;
  // recombination
  const Phase ph_recomb("recombination");
  CK(cudaMemcpyAsync(h->ck.p, kfin.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
  const int tr = tstart(h, kClsRecomb);
  if (recomb == OV_RECOMB_STORED) {
    CK(grow(h->vptr, sizeof(void*) * std::max<size_t>(slots.size(), 1)));
    CK(cudaMemcpyAsync(h->vptr.p, slots.data(), sizeof(void*) * slots.size(), cudaMemcpyHostToDevice, st));
    CK(launch_recombine(h->prec, bt, (const void* const*)h->vptr.p, h->cacc_fin.p, ld, (const int*)h->ck.p,
                        (const double*)h->scale.p, xd, add_x, yd, st));
    h->stats.launches += 1;
    h->stats.other_launches += 1;
  } else {
    // second pass: regenerate t_j from the stored coefficients (ring of two: t_{j+1}
    // overwrites t_{j-1}) and accumulate y += (c_j / nv_j) t_j
    const size_t ab = acc_elem_bytes(h->prec) * pool;
    CK(grow(h->yacc, ab));
    CK(cudaMemsetAsync(h->yacc.p, 0, ab, st));
    CK(cudaMemsetAsync(h->vring.p, 0, 2 * vbn, st));
    CK(launch_pack(h->prec, bt, xd, (char*)h->vring.p + vbn, nullptr, c, (double*)h->partials.p,
                   (unsigned*)h->counters.p, 0, nullptr, st));
    StepArgs b = a;
    b.jdev = nullptr;  // the second pass runs from host-side step indices
    b.slot_tab = nullptr;
    b.yacc = h->yacc.p;
    b.cacc = h->cacc_fin.p;
    for (int jj = 1; jj <= kmax_used; ++jj) {
      b.j = jj;
      b.tc = (char*)h->vring.p + vbn * (jj & 1);
      b.tn = (char*)h->vring.p + vbn * ((jj - 1) & 1);
      b.tp = b.tn;
      CK(launch_step(step_prec(jj), kModeRegen, b, st));
    }
    CK(launch_finish_acc(h->prec, bt, h->yacc.p, (const double*)h->scale.p, xd, add_x, yd, st));
    h->stats.launches += kmax_used + 2;
    h->stats.stencil_launches += kmax_used;
    h->stats.regen_steps += kmax_used;
    h->stats.other_launches += 2;
  }
  tstop(h, tr);
  tstop(h, t_total);
  if (mem == OV_MEM_HOST) CK(cudaMemcpyAsync(y, yd, canon, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  tcollect(h);
  int worst = OV_OK;
  for (int r = 0; r < nrhs; ++r) {
    if (info) {
      info[r].k = kfin[r];
      info[r].l = lfin[r];
      info[r].rh_iters = itfin[r];
      info[r].status = stat[r];
      info[r].err_est = estfin[r];
      info[r].err_inner = estin[r];
    }
    if (stat[r] < 0 && (worst >= 0 || stat[r] < worst)) worst = stat[r];
    else if (worst == OV_OK && stat[r] > 0) worst = stat[r];
  }
  return worst;
}

// With deflation (Sec. 2): sgn(A) x = R sgn(Lambda) (L^dag x) + sgn(A) (I - R L^dag) x, the
// second term by the Krylov path on the deflated source; for A^dag (neg_mu) the roles of R
// and L swap (its eigenvalues are conj(lambda), with the same signs of the real parts).
static int sign_apply_impl(ov_handle* h, int nrhs, const void* x, void* y, int mem, double tol, int k_max, int l,
                           ov_info* info, int add_x, int neg_mu = 0) {
  bool any = false;
  for (const auto& d : h ? h->defl : std::vector<ov_handle::Defl>{}) any = any || d.m > 0;
  if (!h || !any || !x || !y || nrhs < 1) return sign_apply_core(h, nrhs, x, y, mem, tol, k_max, l, info, add_x, neg_mu);
  if (mem != OV_MEM_HOST && mem != OV_MEM_DEVICE) return OV_ERR_ARG;
  if (h->is_batch && nrhs != (int)h->lat.size()) return OV_ERR_ARG;
  CK(cudaSetDevice(h->dev));
  cudaStream_t st = h->st;
  const std::vector<int> lat_of = lattices_of_call(h, nrhs);
  size_t pool = 0;
  for (int q : lat_of) pool += 12 * (size_t)h->lat[q].g.V;
  const size_t vb = sizeof(double2) * pool;
  CK(grow(h->dx, vb));
  CK(grow(h->dy, vb));
  const cudaMemcpyKind kin = mem == OV_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(h->dx.p, x, vb, kin, st));
  // groups of consecutive right-hand sides on one lattice (a single-field handle: one group)
  struct Grp {
    int q, r0, nr;
    size_t off;
  };
  std::vector<Grp> grps;
  size_t off = 0;
  for (int r = 0; r < nrhs; ++r) {
    const int q = lat_of[r];
    if (!grps.empty() && grps.back().q == q && !h->is_batch) ++grps.back().nr;
    else grps.push_back({q, r, 1, off});
    off += 12 * (size_t)h->lat[q].g.V;
  }
  // c = L^dag x per group, x' = x - R c (into dy, the core's source)
  std::vector<std::vector<double2>> coef(grps.size());
  CK(cudaMemcpyAsync(h->dy.p, h->dx.p, vb, cudaMemcpyDeviceToDevice, st));
  for (size_t g = 0; g < grps.size(); ++g) {
    const Grp& G = grps[g];
    const auto& d = h->defl.size() > (size_t)G.q ? h->defl[G.q] : ov_handle::Defl{};
    if (d.m == 0) continue;
    const size_t n = 12 * (size_t)h->lat[G.q].g.V;
    const double2* Rv = (const double2*)(neg_mu ? d.L.p : d.R.p);
    const double2* Lv = (const double2*)(neg_mu ? d.R.p : d.L.p);
    CK(grow(h->dpart, block_gram_part_bytes(d.m, G.nr)));
    CK(grow(h->dG, sizeof(double2) * (size_t)d.m * G.nr * 2));
    double2* Gd = (double2*)h->dG.p;
    const double2* xg = (const double2*)h->dx.p + G.off;
    CK(block_gram(n, Lv, n, d.m, xg, n, G.nr, (double2*)h->dpart.p, Gd, st));
    CK(block_mul(n, Rv, n, d.m, Gd, (double2*)h->dy.p + G.off, n, G.nr, -1.0, 1.0, st));
    coef[g].resize((size_t)d.m * G.nr);
    CK(cudaMemcpyAsync(coef[g].data(), Gd, sizeof(double2) * d.m * G.nr, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  // the Krylov part on the deflated source, in place in dy (its result overwrites it)
  int rc = sign_apply_core(h, nrhs, h->dy.p, h->dx.p, OV_MEM_DEVICE, tol, k_max, l, info, 0, neg_mu, 1);
  if (rc < 0) return rc;
  // y = y' + R sgn(Lambda) c  (and x + gamma5 (...) for the overlap operator)
  for (size_t g = 0; g < grps.size(); ++g) {
    const Grp& G = grps[g];
    const auto& d = h->defl.size() > (size_t)G.q ? h->defl[G.q] : ov_handle::Defl{};
    if (d.m == 0) continue;
    const size_t n = 12 * (size_t)h->lat[G.q].g.V;
    std::vector<double2> cs = coef[g];
    for (int i = 0; i < d.m; ++i) {
      const double sg = d.lam[i].real() >= 0.0 ? 1.0 : -1.0;
      for (int r = 0; r < G.nr; ++r) {
        cs[(size_t)i * G.nr + r].x *= sg;
        cs[(size_t)i * G.nr + r].y *= sg;
      }
    }
    double2* Gd = (double2*)h->dG.p + (size_t)d.m * G.nr;
    CK(cudaMemcpyAsync(Gd, cs.data(), sizeof(double2) * cs.size(), cudaMemcpyHostToDevice, st));
    const double2* Rv = (const double2*)(neg_mu ? d.L.p : d.R.p);
    CK(block_mul(n, Rv, n, d.m, Gd, (double2*)h->dx.p + G.off, n, G.nr, 1.0, 1.0, st));
    CK(cudaStreamSynchronize(st));  // cs is read by the copy before it goes out of scope
  }
  if (add_x) {
    // the source again (dx holds the sign now): from the caller's buffer
    CK(cudaMemcpyAsync(h->dy.p, x, vb, kin, st));
    CK(add_x_gamma5(pool, (const double2*)h->dy.p, (double2*)h->dx.p, st));
  }
  const cudaMemcpyKind kout = mem == OV_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(y, h->dx.p, vb, kout, st));
  CK(cudaStreamSynchronize(st));
  return rc;
}

// for the solver (ov_solve.cu): the sign function on device buffers, of A (neg_mu = 0) or
// of A^dag = gamma5 D_w(-mu) (neg_mu = 1)
int ov::sign_apply_device(ov_handle* h, int nrhs, const double2* x, double2* y, double tol, int k_max, int l,
                          ov_info* info, int neg_mu) {
  return sign_apply_impl(h, nrhs, x, y, OV_MEM_DEVICE, tol, k_max, l, info, 0, neg_mu);
}
cudaStream_t ov::handle_stream(const ov_handle* h) { return h->st; }
size_t ov::lattice_size(const ov_handle* h, int q) { return 12 * (size_t)h->lat[q].g.V; }
double ov::lattice_mu(const ov_handle* h, int q) { return h->lat[q].mu; }
double ov::lattice_mass(const ov_handle* h, int q) { return h->lat[q].m_w + 4.0; }

// A fixed set of matvecs (one per item: lattice, sign of mu, offset of the vector in the
// canonical block buffers), its problem descriptors and block map uploaded once; every run
// is one pack, one stencil launch and one unpack over all items.
struct ov::ApplySet {
  Buf desc, map;
  Batch bt{};
  size_t pool = 0;
  int nitems = 0, maxblk = 0;
};

int ov::apply_set_create(ov_handle* h, const std::vector<ApplyItem>& items, size_t pool, ApplySet** out) {
  *out = nullptr;
  if (items.empty()) return OV_ERR_ARG;
  const int bs = h->o.block_size ? h->o.block_size : kBlockDefault;
  const int np = (int)items.size();
  std::vector<ProbDesc> d(np);
  std::vector<int2> map;
  int blk = 0, maxblk = 0;
  bool same = true;
  for (int r = 0; r < np; ++r) {
    const ApplyItem& it = items[r];
    if (it.q < 0 || it.q >= (int)h->lat.size() || it.voff + 12 * (size_t)h->lat[it.q].g.V > pool) return OV_ERR_ARG;
    const Lattice& L = h->lat[it.q];
    d[r].g = L.g;
    d[r].links = L.links.p;
    fill_consts(d[r], L.m_w, it.neg ? -L.mu : L.mu);
    d[r].voff = it.voff;
    d[r].block0 = blk;
    d[r].nblk = num_site_blocks(L.g, bs);
    blk += d[r].nblk;
    maxblk += num_site_blocks(L.g, 64);
    same = same && it.q == items[0].q;
  }
  // as build_batch: site-block-major for one lattice (the items share links in L2)
  if (same) {
    for (int qb = 0; qb < d[0].nblk; ++qb)
      for (int r = 0; r < np; ++r) map.push_back(make_int2(r, qb));
  } else {
    for (int r = 0; r < np; ++r)
      for (int qb = 0; qb < d[r].nblk; ++qb) map.push_back(make_int2(r, qb));
  }
  ApplySet* a = new ApplySet;
  if (grow(a->desc, sizeof(ProbDesc) * np) != cudaSuccess || grow(a->map, sizeof(int2) * map.size()) != cudaSuccess) {
    apply_set_destroy(a);
    return OV_ERR_NOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(a->desc.p, d.data(), sizeof(ProbDesc) * np, cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(a->map.p, map.data(), sizeof(int2) * map.size(), cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);  // the host vectors go out of scope
  if (e != cudaSuccess) {
    apply_set_destroy(a);
    return OV_ERR_CUDA;
  }
  a->bt.desc = (const ProbDesc*)a->desc.p;
  a->bt.blk_map = (const int2*)a->map.p;
  a->bt.nblocks = blk;
  a->bt.nprob = np;
  a->bt.block = bs;
  a->pool = pool;
  a->nitems = np;
  a->maxblk = maxblk;
  *out = a;
  return OV_OK;
}

void ov::apply_set_destroy(ApplySet* a) {
  if (!a) return;
  release(a->desc);
  release(a->map);
  delete a;
}

int ov::apply_set_run(ov_handle* h, const ApplySet* a, const double2* X, double2* Y) {
  cudaStream_t st = h->st;
  int rc = ensure_outer(h, std::max(a->nitems, h->cap_rhs), std::max(h->cap_ld, 4), a->pool, a->maxblk);
  if (rc != OV_OK) return rc;
  Coefs c = coefs(h, h->cap_ld);
  CK(launch_pack(h->prec, a->bt, X, h->tv.p, nullptr, c, (double*)h->partials.p, (unsigned*)h->counters.p, 0, nullptr,
                 st));
  StepArgs sa{};
  sa.b = a->bt;
  sa.tv = h->tv.p;
  sa.p = h->p.p;
  sa.dagger = 0;
  sa.c = c;
  CK(launch_step(h->prec, kModeApply, sa, st));
  CK(launch_unpack(h->prec, a->bt, h->p.p, Y, st));
  h->stats.launches += 3;
  h->stats.stencil_launches += 1;
  h->stats.other_launches += 2;
  return OV_OK;
}

extern "C" int ov_deflate(ov_handle* h, int m, double tol, int maxit, double* lam_out, double* res_out, int* m_used) {
  if (!h || m < 0 || !(tol > 0.0) || maxit < 1) return OV_ERR_ARG;
  if (m > 48) return OV_ERR_TOO_LARGE;
  CK(cudaSetDevice(h->dev));
  const Phase ph("ov_deflate");
  const int nl = (int)h->lat.size();
  for (int q = 0; q < nl; ++q)
    if ((size_t)2 * m + 8 > 12 * (size_t)h->lat[q].g.V && m > 0) return OV_ERR_ARG;
  h->defl.resize(nl);
  for (int q = 0; q < nl; ++q) {
    h->defl[q].m = 0;
    if (m_used) m_used[q] = 0;
  }
  if (m == 0) {
    for (auto& d : h->defl) {
      release(d.R);
      release(d.L);
    }
    return OV_OK;
  }
  // a block of 2 m + 8 vectors: the filter's gap is between the m-th and the b-th eigenvalue
  const int b = std::min<int>(64, 2 * m + 8);
  const int deg = 48;  // the filter's largest degree (ov_eig.cu lowers it while the cut is high)
  // one job per lattice for the right eigenvectors, one more at mu != 0 for the left ones
  // (right eigenvectors of A^dag = A(-mu) for conj(lambda)); all jobs run together
  std::vector<Buf> R0(nl), L0(nl);
  std::vector<EigJob> jobs;
  std::vector<int> jr(nl, -1), jl(nl, -1);
  size_t nmax = 0;
  Buf tmp, part, g;
  auto cleanup = [&]() {
    for (int q = 0; q < nl; ++q) {
      release(R0[q]);
      release(L0[q]);
    }
    release(tmp);
    release(part);
    release(g);
  };
  for (int q = 0; q < nl; ++q) {
    const size_t n = 12 * (size_t)h->lat[q].g.V;
    nmax = std::max(nmax, n);
    if (grow(R0[q], sizeof(double2) * n * m) != cudaSuccess) {
      cleanup();
      return OV_ERR_NOMEM;
    }
    EigJob jb;
    jb.q = q;
    jb.Rout = (double2*)R0[q].p;
    jr[q] = (int)jobs.size();
    jobs.push_back(jb);
    if (h->lat[q].mu != 0.0) {
      if (grow(L0[q], sizeof(double2) * n * m) != cudaSuccess) {
        cleanup();
        return OV_ERR_NOMEM;
      }
      jb.neg = 1;
      jb.Rout = (double2*)L0[q].p;
      jl[q] = (int)jobs.size();
      jobs.push_back(jb);
    }
  }
  if (grow(tmp, sizeof(double2) * nmax * m) != cudaSuccess || grow(part, block_gram_part_bytes(m, m)) != cudaSuccess ||
      grow(g, sizeof(double2) * m * m) != cudaSuccess) {
    cleanup();
    return OV_ERR_NOMEM;
  }
  const int erc = eig_smallest(h, jobs, m, b, deg, tol, maxit, h->trace);
  if (erc < 0) {
    cleanup();
    return erc;
  }
  int worst = OV_OK;
  for (int q = 0; q < nl; ++q) {
    auto& d = h->defl[q];
    const size_t n = 12 * (size_t)h->lat[q].g.V;
    const bool herm = jl[q] < 0;
    std::vector<std::complex<double>> lam = jobs[jr[q]].lam;
    std::vector<double> res = jobs[jr[q]].res;
    std::vector<int> perm(m);
    for (int i = 0; i < m; ++i) perm[i] = i;
    if (!herm) {
      // left eigenvectors matched to the right ones by eigenvalue
      const auto& lamL = jobs[jl[q]].lam;
      const auto& resL = jobs[jl[q]].res;
      std::vector<int> used(m, 0);
      for (int i = 0; i < m; ++i) {
        int best = 0;
        double bd = INFINITY;
        for (int j = 0; j < m; ++j) {
          const double dd = std::abs(lamL[j] - std::conj(lam[i]));
          if (!used[j] && dd < bd) { bd = dd; best = j; }
        }
        used[best] = 1;
        perm[i] = best;
        // a pair counts as converged only when both sides are and the eigenvalues agree
        res[i] = std::max(std::max(res[i], resL[best]), bd / std::max(std::abs(lam[i]), 1e-300) * 1e-3);
      }
    }
    // keep the converged pairs only: the deflation formula is exact for any set of true
    // eigenpairs, while an inaccurate pair would put its error into the exact part
    std::vector<int> keep;
    for (int i = 0; i < m; ++i)
      if (res[i] <= tol) keep.push_back(i);
    const int mk = (int)keep.size();
    if (mk < m) worst = OV_NOT_CONVERGED;
    if (grow(d.R, sizeof(double2) * n * std::max(mk, 1)) != cudaSuccess ||
        grow(d.L, sizeof(double2) * n * std::max(mk, 1)) != cudaSuccess) {
      cleanup();
      return OV_ERR_NOMEM;
    }
    if (mk > 0) {
      std::vector<double2> C((size_t)m * mk, make_double2(0.0, 0.0));
      for (int c = 0; c < mk; ++c) C[(size_t)keep[c] * mk + c] = make_double2(1.0, 0.0);
      cudaError_t e = cudaMemcpyAsync(g.p, C.data(), sizeof(double2) * m * mk, cudaMemcpyHostToDevice, h->st);
      if (e == cudaSuccess)
        e = block_mul(n, (double2*)R0[q].p, n, m, (double2*)g.p, (double2*)d.R.p, n, mk, 1.0, 0.0, h->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
      if (e != cudaSuccess) {
        cleanup();
        return OV_ERR_CUDA;
      }
      if (herm) {
        e = cudaMemcpyAsync(d.L.p, d.R.p, sizeof(double2) * n * mk, cudaMemcpyDeviceToDevice, h->st);
      } else {
        // L <- L (L^dag R)^{-dag} on the kept pairs, so that L^dag R = 1
        std::fill(C.begin(), C.end(), make_double2(0.0, 0.0));
        for (int c = 0; c < mk; ++c) C[(size_t)perm[keep[c]] * mk + c] = make_double2(1.0, 0.0);
        std::vector<double2> M((size_t)mk * mk), Mi((size_t)mk * mk);
        e = cudaMemcpyAsync(g.p, C.data(), sizeof(double2) * m * mk, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess)
          e = block_mul(n, (double2*)L0[q].p, n, m, (double2*)g.p, (double2*)tmp.p, n, mk, 1.0, 0.0, h->st);
        if (e == cudaSuccess)
          e = block_gram(n, (double2*)tmp.p, n, mk, (double2*)d.R.p, n, mk, (double2*)part.p, (double2*)g.p, h->st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(M.data(), g.p, sizeof(double2) * mk * mk, cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess || !small_inv(mk, M.data(), Mi.data())) {
          cleanup();
          return e != cudaSuccess ? OV_ERR_CUDA : OV_ERR_BREAKDOWN;
        }
        std::vector<double2> Ci((size_t)mk * mk);
        for (int i = 0; i < mk; ++i)
          for (int j = 0; j < mk; ++j)
            Ci[(size_t)i * mk + j] = make_double2(Mi[(size_t)j * mk + i].x, -Mi[(size_t)j * mk + i].y);  // Minv^dag
        e = cudaMemcpyAsync(g.p, Ci.data(), sizeof(double2) * mk * mk, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess)
          e = block_mul(n, (double2*)tmp.p, n, mk, (double2*)g.p, (double2*)d.L.p, n, mk, 1.0, 0.0, h->st);
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
      if (e != cudaSuccess) {
        cleanup();
        return OV_ERR_CUDA;
      }
    }
    d.m = mk;
    d.lam.clear();
    d.res.clear();
    for (int c = 0; c < mk; ++c) {
      d.lam.push_back(lam[keep[c]]);
      d.res.push_back(res[keep[c]]);
    }
    if (m_used) m_used[q] = mk;
    for (int i = 0; i < m; ++i) {
      if (lam_out) {
        lam_out[2 * ((size_t)q * m + i)] = lam[i].real();
        lam_out[2 * ((size_t)q * m + i) + 1] = lam[i].imag();
      }
      if (res_out) res_out[(size_t)q * m + i] = res[i];
    }
  }
  cleanup();
  return worst;
}

extern "C" int ov_get_deflation(const ov_handle* h, int lattice, int mcap, void* lam, void* R, void* L, int* m) {
  if (!h || lattice < 0 || lattice >= (int)h->lat.size() || mcap < 0) return OV_ERR_ARG;
  CK(cudaSetDevice(h->dev));
  const int md = lattice < (int)h->defl.size() ? h->defl[lattice].m : 0;
  const int mm = std::min(mcap, md);
  if (m) *m = mm;
  if (mm == 0) return OV_OK;
  const auto& d = h->defl[lattice];
  const size_t n = 12 * (size_t)h->lat[lattice].g.V;
  if (lam)
    for (int i = 0; i < mm; ++i) ((double2*)lam)[i] = make_double2(d.lam[i].real(), d.lam[i].imag());
  if (R) CK(cudaMemcpy(R, d.R.p, sizeof(double2) * n * mm, cudaMemcpyDeviceToHost));
  if (L) CK(cudaMemcpy(L, d.L.p, sizeof(double2) * n * mm, cudaMemcpyDeviceToHost));
  return OV_OK;
}
int ov::handle_device(const ov_handle* h) { return h->dev; }
size_t ov::handle_pool(const ov_handle* h, int nrhs) {
  if (h->is_batch) {
    size_t n = 0;
    for (const Lattice& L : h->lat) n += 12 * (size_t)L.g.V;
    return nrhs == (int)h->lat.size() ? n : 0;
  }
  return 12 * (size_t)h->lat[0].g.V * nrhs;
}

extern "C" int ov_sign_apply(ov_handle* h, int nrhs, const void* x, void* y, int mem, double tol, int k_max, int l,
                             ov_info* info) {
  return sign_apply_impl(h, nrhs, x, y, mem, tol, k_max, l, info, 0);
}

extern "C" int ov_apply(ov_handle* h, int nrhs, const void* x, void* y, int mem, double tol, int k_max, int l,
                        ov_info* info) {
  return sign_apply_impl(h, nrhs, x, y, mem, tol, k_max, l, info, 1);
}

// ---------------------------------------------------------------- stencil alone
extern "C" int ov_wilson_apply(ov_handle* h, int nrhs, const void* x, void* y, int mem, int dagger) {
  if (!h || !x || !y || nrhs < 1) return OV_ERR_ARG;
  if (mem != OV_MEM_HOST && mem != OV_MEM_DEVICE) return OV_ERR_ARG;
  if (h->is_batch && nrhs != (int)h->lat.size()) return OV_ERR_ARG;
  CK(cudaSetDevice(h->dev));
  cudaStream_t st = h->st;
  Batch bt;
  size_t pool = 0;
  const std::vector<int> lat_of = lattices_of_call(h, nrhs);
  int rc = build_batch(h, lat_of, h->o.block_size ? h->o.block_size : kBlockDefault, &bt, &pool);
  if (rc != OV_OK) return rc;
  rc = ensure_outer(h, nrhs, std::max(h->cap_ld, 4), pool, max_blocks(h, lat_of));
  if (rc != OV_OK) return rc;
  const size_t canon = sizeof(double2) * pool;
  const double2* xd = (const double2*)x;
  double2* yd = (double2*)y;
  if (mem == OV_MEM_HOST) {
    CK(grow(h->xcanon, canon));
    CK(grow(h->ycanon, canon));
    CK(cudaMemcpyAsync(h->xcanon.p, x, canon, cudaMemcpyHostToDevice, st));
    xd = (const double2*)h->xcanon.p;
    yd = (double2*)h->ycanon.p;
  }
  Coefs c = coefs(h, h->cap_ld);
  CK(launch_pack(h->prec, bt, xd, h->tv.p, nullptr, c, (double*)h->partials.p, (unsigned*)h->counters.p, 0, nullptr,
                 st));
  StepArgs a{};
  a.b = bt;
  a.tv = h->tv.p;
  a.p = h->p.p;
  a.dagger = dagger ? 1 : 0;
  a.c = c;
  CK(launch_step(h->prec, kModeApply, a, st));
  CK(launch_unpack(h->prec, bt, h->p.p, yd, st));
  h->stats.launches += 3;
  h->stats.stencil_launches += 1;
  h->stats.other_launches += 2;
  if (mem == OV_MEM_HOST) CK(cudaMemcpyAsync(y, yd, canon, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return OV_OK;
}

// ---------------------------------------------------------------- batch of lattices
extern "C" int ov_batch_create(ov_handle** hp, int nprob, const ov_geom* geoms, const void* const* links, int links_mem,
                               const double* m_w, const double* mu, const ov_opts* opts, void* stream) {
  if (!hp || nprob < 1 || !geoms || !links || !m_w || !mu) return OV_ERR_ARG;
  *hp = nullptr;
  ov_handle* first = nullptr;
  int rc = ov_create(&first, &geoms[0], links[0], links_mem, m_w[0], mu[0], opts, stream);
  if (rc != OV_OK) return rc;
  for (int i = 1; i < nprob; ++i) {
    if (geoms[i].precision != geoms[0].precision || (geoms[i].t_antiperiodic != 0) != (geoms[0].t_antiperiodic != 0)) {
      ov_destroy(first);
      return OV_ERR_ARG;
    }
    ov_handle* hi = nullptr;
    rc = ov_create(&hi, &geoms[i], links[i], links_mem, m_w[i], mu[i], opts, stream);
    if (rc != OV_OK) {
      ov_destroy(first);
      return rc;
    }
    // move the converted links into the batch handle
    first->lat.push_back(hi->lat[0]);
    hi->lat[0].links = Buf{};
    ov_destroy(hi);
  }
  first->is_batch = 1;
  *hp = first;
  return OV_OK;
}

extern "C" int ov_batch_sign_apply(ov_handle* h, const void* const* x, void* const* y, int mem, double tol, int k_max,
                                   int l, ov_info* info) {
  if (!h || !h->is_batch || !x || !y) return OV_ERR_ARG;
  if (mem != OV_MEM_HOST && mem != OV_MEM_DEVICE) return OV_ERR_ARG;
  CK(cudaSetDevice(h->dev));
  const int np = (int)h->lat.size();
  size_t pool = 0;
  for (const Lattice& L : h->lat) pool += 12 * (size_t)L.g.V;
  Buf xb, yb;
  if (grow(xb, sizeof(double2) * pool) != cudaSuccess || grow(yb, sizeof(double2) * pool) != cudaSuccess) {
    release(xb);
    release(yb);
    return OV_ERR_NOMEM;
  }
  const cudaMemcpyKind kin = mem == OV_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind kout = mem == OV_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  size_t off = 0;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < np && e == cudaSuccess; ++r) {
    const size_t nb = sizeof(double2) * 12 * (size_t)h->lat[r].g.V;
    e = cudaMemcpyAsync((char*)xb.p + off, x[r], nb, kin, h->st);
    off += nb;
  }
  int rc = e == cudaSuccess ? sign_apply_impl(h, np, xb.p, yb.p, OV_MEM_DEVICE, tol, k_max, l, info, 0) : OV_ERR_CUDA;
  if (rc >= 0) {
    off = 0;
    for (int r = 0; r < np && e == cudaSuccess; ++r) {
      const size_t nb = sizeof(double2) * 12 * (size_t)h->lat[r].g.V;
      e = cudaMemcpyAsync(y[r], (char*)yb.p + off, nb, kout, h->st);
      off += nb;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) rc = OV_ERR_CUDA;
  }
  release(xb);
  release(yb);
  return rc;
}

// ---------------------------------------------------------------- inner level alone
extern "C" int ov_inner_sign(ov_handle* h, int count, int ld, const int* k, const void* alpha, const void* beta,
                             const void* gamma, int hermitian, int l, void* cout, double* est_inner, int* rh_iters) {
  if (!h || count < 1 || !k || !alpha || !beta || !gamma || !cout || l < 1) return OV_ERR_ARG;
  if (ld < 1) return OV_ERR_ARG;
  if (l > kMaxL || ld > kMaxInnerK) return OV_ERR_TOO_LARGE;
  for (int i = 0; i < count; ++i)
    if (k[i] < 1 || k[i] > ld) return OV_ERR_ARG;
  CK(cudaSetDevice(h->dev));
  cudaStream_t st = h->st;
  const int ldi = ld + 2;
  int rc = ensure_inner(h, count, ldi);
  if (rc != OV_OK) return rc;
  // coefficients in the 1-based layout of the outer level
  std::vector<double2> A((size_t)count * ldi), B((size_t)count * ldi), G((size_t)count * ldi);
  const double2* ai = (const double2*)alpha;
  const double2* bi = (const double2*)beta;
  const double2* gi = (const double2*)gamma;
  for (int i = 0; i < count; ++i)
    for (int jj = 0; jj < ld; ++jj) {
      A[(size_t)i * ldi + jj + 1] = ai[(size_t)i * ld + jj];
      B[(size_t)i * ldi + jj + 1] = bi[(size_t)i * ld + jj];
      G[(size_t)i * ldi + jj + 1] = hermitian ? bi[(size_t)i * ld + jj] : gi[(size_t)i * ld + jj];
    }
  Buf dA, dB, dG;
  auto cleanup = [&]() {
    release(dA);
    release(dB);
    release(dG);
  };
  const size_t cb = sizeof(double2) * (size_t)count * ldi;
  if (grow(dA, cb) != cudaSuccess || grow(dB, cb) != cudaSuccess || grow(dG, cb) != cudaSuccess) {
    cleanup();
    return OV_ERR_NOMEM;
  }
  std::vector<int> lv(count, l);
  cudaMemcpyAsync(dA.p, A.data(), cb, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dB.p, B.data(), cb, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dG.p, G.data(), cb, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->ck.p, k, sizeof(int) * count, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->cl.p, lv.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st);
  InnerWork iw = inner_work(h);
  cudaError_t e = run_inner(count, (const int*)h->ck.p, (const int*)h->cl.p, hermitian ? 1 : 0, (double2*)dA.p,
                            (double2*)dB.p, (double2*)dG.p, nullptr, ldi, iw, h->o.rh_tol, h->o.rh_maxit, h->o.inner_dl,
                            (double2*)h->cc_cur.p, ldi, nullptr, h->prec, (double*)h->c_est_in.p, nullptr, ldi,
                            nullptr, nullptr, (int*)h->c_rhst.p, (int*)h->c_rhit.p, 0, st);
  std::vector<double2> C((size_t)count * ldi);
  std::vector<double> ein(count);
  std::vector<int> rs(count), ri(count);
  if (e == cudaSuccess) e = cudaMemcpyAsync(C.data(), h->cc_cur.p, cb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ein.data(), h->c_est_in.p, sizeof(double) * count, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rs.data(), h->c_rhst.p, sizeof(int) * count, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ri.data(), h->c_rhit.p, sizeof(int) * count, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) {
    fprintf(stderr, "libov: ov_inner_sign: %s\n", cudaGetErrorString(e));
    return OV_ERR_CUDA;
  }
  double2* co = (double2*)cout;
  int worst = OV_OK;
  for (int i = 0; i < count; ++i) {
    for (int jj = 0; jj < ld; ++jj) co[(size_t)i * ld + jj] = jj < k[i] ? C[(size_t)i * ldi + jj + 1] : double2{0, 0};
    if (est_inner) est_inner[i] = ein[i];
    if (rh_iters) rh_iters[i] = ri[i];
    if (rs[i] != 0) worst = OV_ERR_RH_NOCONV;
  }
  return worst;
}

extern "C" int ov_rh_sign(ov_handle* h, int count, int m, const void* T, void* S, int* iters) {
  if (!h || count < 1 || m < 1 || !T || !S) return OV_ERR_ARG;
  if (m > kMaxInnerK) return OV_ERR_TOO_LARGE;
  CK(cudaSetDevice(h->dev));
  cudaStream_t st = h->st;
  if (m > kMaxL) {
    // beyond one CTA's shared memory: Gauss-Jordan over global memory, FP64
    const size_t mb = sizeof(double2) * (size_t)count * m * m;
    Buf dT, dS, scr;
    auto cleanup = [&]() {
      release(dT);
      release(dS);
      release(scr);
    };
    if (grow(dT, mb) != cudaSuccess || grow(dS, mb) != cudaSuccess ||
        grow(scr, rh_big_scratch_bytes(count, m)) != cudaSuccess) {
      cleanup();
      return OV_ERR_NOMEM;
    }
    std::vector<int> it(count), ok(count);
    cudaError_t e = cudaMemcpyAsync(dT.p, T, mb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = run_rh_big(count, m, (const double2*)dT.p, (double2*)dS.p, it.data(), ok.data(), h->o.rh_tol, h->o.rh_maxit,
                     scr.p, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S, dS.p, mb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) {
      fprintf(stderr, "libov: ov_rh_sign: %s\n", cudaGetErrorString(e));
      return OV_ERR_CUDA;
    }
    int worst = OV_OK;
    for (int i = 0; i < count; ++i) {
      if (iters) iters[i] = it[i];
      if (!ok[i]) worst = OV_ERR_RH_NOCONV;
    }
    return worst;
  }
  int rc = ensure_inner(h, (count + 1) / 2, std::max(h->inner_ld, 4));
  if (rc != OV_OK) return rc;
  const size_t mb = sizeof(double2) * (size_t)count * m * m;
  Buf dT, dS, dI;
  auto cleanup = [&]() {
    release(dT);
    release(dS);
    release(dI);
  };
  if (grow(dT, mb) != cudaSuccess || grow(dS, mb) != cudaSuccess || grow(dI, sizeof(int) * 2 * count) != cudaSuccess) {
    cleanup();
    return OV_ERR_NOMEM;
  }
  InnerWork iw = inner_work(h);
  cudaError_t e = cudaMemcpyAsync(dT.p, T, mb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = run_rh_dense(count, m, (const double2*)dT.p, (double2*)dS.p, (int*)dI.p, (int*)dI.p + count, h->o.rh_tol,
                     h->o.rh_maxit, iw, st);
  std::vector<int> it(2 * count);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S, dS.p, mb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(it.data(), dI.p, sizeof(int) * 2 * count, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) {
    fprintf(stderr, "libov: ov_rh_sign: %s\n", cudaGetErrorString(e));
    return OV_ERR_CUDA;
  }
  int worst = OV_OK;
  for (int i = 0; i < count; ++i) {
    if (iters) iters[i] = it[i];
    if (!it[count + i]) worst = OV_ERR_RH_NOCONV;
  }
  return worst;
}

extern "C" int ov_set_sizer(ov_handle* h, const float* theta, int l_min, int l_max) {
  if (!h) return OV_ERR_ARG;
  if (!theta) {
    h->sizer_on = 0;
    return OV_OK;
  }
  if (l_min < 1 || l_max < l_min) return OV_ERR_ARG;
  if (l_max > kMaxL) return OV_ERR_TOO_LARGE;
  CK(cudaSetDevice(h->dev));
  const size_t nb = sizeof(float) * mlp_num_params();
  CK(grow(h->sizer_theta, nb));
  CK(cudaMemcpy(h->sizer_theta.p, theta, nb, cudaMemcpyHostToDevice));
  h->sizer_lmin = l_min;
  h->sizer_lmax = l_max;
  h->sizer_on = 1;
  return OV_OK;
}

extern "C" int ov_get_coefficients(const ov_handle* h, int rhs, int kcap, void* alpha, void* beta, void* gamma,
                                   int* k) {
  if (!h || !alpha || !beta || !gamma || kcap < 1) return OV_ERR_ARG;
  if (rhs < 0 || rhs >= h->last_nrhs || h->last_steps < 1) return OV_ERR_ARG;
  CK(cudaSetDevice(h->dev));
  const int kk = std::min(kcap, h->last_steps);
  const size_t o = (size_t)rhs * h->last_ld + 1;
  // alpha_1..alpha_k, beta_1..beta_k (beta_1 = 0), gamma_1..gamma_k
  CK(cudaMemcpy(alpha, (const double2*)h->coef_alp.p + o, sizeof(double2) * kk, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(beta, (const double2*)h->coef_bet.p + o, sizeof(double2) * kk, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(gamma, (const double2*)h->coef_gam.p + o, sizeof(double2) * kk, cudaMemcpyDeviceToHost));
  if (k) *k = kk;
  return OV_OK;
}

extern "C" int ov_version(char* buf, size_t len) {
  if (!buf || len == 0) return OV_ERR_ARG;
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    snprintf(buf, len, "libov 0.1 (no device)");
    return OV_ERR_CUDA;
  }
  snprintf(buf, len, "libov 0.1 sm_%d%d %s", p.major, p.minor, p.name);
  return OV_OK;
}
