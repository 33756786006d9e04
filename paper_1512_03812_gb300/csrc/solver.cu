// solver.cu -- batched conjugate gradient on D^dag D x = b.
//
// The paper does not name its solver for the inversions of D (Sec. 3, end);
// CG on the normal operator is used.  All chains of the batch iterate in the
// same launches; each chain carries its own scalars (CgChain) and leaves the
// iteration when it converges: its blocks then exit at once.
//
// One iteration is two kernels:
//   A: p <- r + beta p (recomputed at the four neighbours, so no extra pass),
//      t <- D p, and |t|^2 = p^dag D^dag D p  ->  alpha = |r|^2 / |t|^2
//   B: A p = D^dag t, x <- x + alpha p, r <- r - alpha A p, |r|^2 -> beta
// Two search-direction buffers alternate; each chain records which one holds
// its p, so kernel arguments never change between iterations.
//
// SM_F64: FP64 fields; the chain stops when |r| <= tol |b| for the recursive
// residual, and the FP64 true residual is reported at the end.
// SM_MIXED: FP32 fields for x, r, p, t and FP32 links; reliable updates
// (Sleijpen and van der Vorst; in the mixed-precision form of Clark et al.,
// 2010) fold the FP32 solution into the FP64 x and replace r by the FP64 true
// residual b - A x whenever |r| has fallen by `delta` since the last update,
// and when the FP32 residual meets the tolerance.  The chain stops when the
// FP64 true residual meets it.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sm {

#define SM_CU(call)                                                                           \
  do {                                                                                        \
    const cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(SM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename R>
struct CgArgs {
  const R* U;        // links in the iteration precision
  const double* U64; // FP64 links (reliable updates, true residual)
  const double* b;
  R* r;
  R* x;              // iterate: the solution (F64) or its FP32 correction (MIXED)
  R* pa;
  R* pb;
  R* t;
  double* xhi;       // FP64 solution (MIXED)
  double* t64;       // FP64 scratch (reliable updates)
  CgChain* cgc;
  double* partials;
  unsigned* counters;
  int* n_active;  // [0] chains still iterating, [1] chains due a reliable update
  double tol2, delta2;
  int maxit;
  int mixed;
  const unsigned char* grid_mask;  // if set, only chains with mask 1 take the grid path
};

#define CHAIN_PROLOGUE                     \
  const int c_ = g.blk_chain[blockIdx.x];  \
  const ChainInfo ci = g.chains[c_];       \
  CgChain* cc = a.cgc + c_;

template <typename R>
__device__ __forceinline__ Sp<R> to_r(Sp<double> v) {
  return {{(R)v.a.re, (R)v.a.im}, {(R)v.b.re, (R)v.b.im}};
}
__device__ __forceinline__ Sp<double> to_d(Sp<float> v) {
  return {{v.a.re, v.a.im}, {v.b.re, v.b.im}};
}
__device__ __forceinline__ Sp<double> to_d(Sp<double> v) { return v; }

// r = b, x = 0, p = 0, |b|^2 -> the chain's scalars.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_cg_init(Geo g, CgArgs<R> a) {
  CHAIN_PROLOGUE
  if (a.grid_mask && !a.grid_mask[c_]) return;  // solved by the chain-resident kernel
  const Site s = site_of(g, ci, c_);
  double v[1] = {0.0};
  if (s.valid) {
    const Sp<double> bv = ld_sp(a.b, s.n);
    v[0] = norm2(bv);
    const Sp<R> z = {{0, 0}, {0, 0}};
    st_sp(a.r, s.n, to_r<R>(bv));
    st_sp(a.x, s.n, z);
    st_sp(a.pa, s.n, z);
    if (a.mixed) st_sp(a.xhi, s.n, Sp<double>{{0, 0}, {0, 0}});
  }
  double tot[1];
  if (chain_reduce<1>(v, a.partials, a.counters, g, ci, c_, tot) && threadIdx.x == 0) {
    const double bb = tot[0];
    cc->bb = bb;
    cc->rr = cc->rr_prev = cc->rmax = cc->rr_true = bb;
    cc->alpha = cc->beta = 0.0;
    cc->iters = 0;
    cc->par = 0;
    cc->need_update = 0;
    cc->updates = 0;
    cc->alpha_x = 0.0;
    cc->flags = 0;
    if (bb > 0.0 && isfinite(bb)) {
      cc->state = 1;
      atomicAdd(a.n_active, 1);
    } else {
      cc->state = 0;
      if (!isfinite(bb)) cc->flags |= 2;
    }
  }
}

// Kernel A: p <- r + beta p at n and its neighbours; t = D p; alpha.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_cg_a(Geo g, CgArgs<R> a) {
  CHAIN_PROLOGUE
  if (cc->state != 1) return;
  const Site s = site_of(g, ci, c_);
  const int par = cc->par;
  const R beta = (R)cc->beta;
  const R* __restrict__ pold = par ? a.pb : a.pa;
  R* __restrict__ pnew = par ? a.pa : a.pb;
  double v[1] = {0.0};
  if (s.valid) {
    auto P = [&](long long m) { return ld_sp(a.r, m) + beta * ld_sp(pold, m); };
    const long long nxm = at(s, xm1(s), s.t), ntm = at(s, s.x, tm1(s));
    const Sp<R> p0 = P(s.n);
    st_sp(pnew, s.n, p0);
    const Lk<R> u = ld_lk(a.U, s.n);
    const Sp<R> o = hop_sum<false, R>(P(at(s, xp1(s), s.t)), P(nxm), P(at(s, s.x, tp1(s))), P(ntm),
                                      u.x, ld_lk(a.U, nxm).x, u.t, ld_lk(a.U, ntm).t);
    const Sp<R> tv = (R)(2.0 + ci.m0) * p0 - (R)0.5 * o;
    st_sp(a.t, s.n, tv);
    v[0] = (double)norm2(tv);
  }
  double tot[1];
  if (chain_reduce<1>(v, a.partials, a.counters, g, ci, c_, tot) && threadIdx.x == 0) {
    const double pAp = tot[0];
    if (pAp > 0.0 && isfinite(pAp)) {
      cc->alpha = cc->rr / pAp;
    } else {  // breakdown: leave the chain with its current iterate
      cc->alpha = 0.0;
      cc->flags |= 2;
      cc->state = 0;
      atomicSub(a.n_active, 1);
    }
  }
}

// Kernel B: A p = D^dag t; x += alpha p; r -= alpha A p; beta; convergence.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_cg_b(Geo g, CgArgs<R> a) {
  CHAIN_PROLOGUE
  if (cc->state != 1) return;
  const Site s = site_of(g, ci, c_);
  const R* __restrict__ pnew = cc->par ? a.pa : a.pb;
  const R alpha = (R)cc->alpha;
  double v[1] = {0.0};
  if (s.valid) {
    const long long nxm = at(s, xm1(s), s.t), ntm = at(s, s.x, tm1(s));
    const Lk<R> u = ld_lk(a.U, s.n);
    const Sp<R> o = hop_sum<true, R>(ld_sp(a.t, at(s, xp1(s), s.t)), ld_sp(a.t, nxm),
                                     ld_sp(a.t, at(s, s.x, tp1(s))), ld_sp(a.t, ntm), u.x,
                                     ld_lk(a.U, nxm).x, u.t, ld_lk(a.U, ntm).t);
    const Sp<R> Ap = (R)(2.0 + ci.m0) * ld_sp(a.t, s.n) - (R)0.5 * o;
    const Sp<R> pv = ld_sp(pnew, s.n);
    st_sp(a.x, s.n, ld_sp_cg(a.x, s.n) + alpha * pv);
    const Sp<R> rv = ld_sp_cg(a.r, s.n) - alpha * Ap;
    st_sp(a.r, s.n, rv);
    v[0] = (double)norm2(rv);
  }
  double tot[1];
  if (chain_reduce<1>(v, a.partials, a.counters, g, ci, c_, tot) && threadIdx.x == 0) {
    const double rr = tot[0];
    cc->rr_prev = cc->rr;
    cc->rr = rr;
    cc->beta = rr / cc->rr_prev;
    cc->par ^= 1;
    cc->iters += 1;
    const bool conv = rr <= a.tol2 * cc->bb;
    if (!isfinite(rr)) {
      cc->flags |= 2;
      cc->state = 0;
      atomicSub(a.n_active, 1);
    } else if (a.mixed) {
      if (conv || cc->iters >= a.maxit) {
        cc->state = 2;  // wait for the FP64 check
        mark_update(cc, a.n_active + 1);
      } else if (rr < a.delta2 * cc->rmax) {
        mark_update(cc, a.n_active + 1);
      }
      cc->rmax = fmax(cc->rmax, rr);
    } else if (conv) {
      cc->state = 0;
      atomicSub(a.n_active, 1);
    } else if (cc->iters >= a.maxit) {
      cc->flags |= 1;
      cc->state = 0;
      atomicSub(a.n_active, 1);
    }
  }
}

// FP64 residual, step 1: t64 = D (xhi + x), for chains that asked for a
// reliable update (all chains if `all`).  x may be NULL.
__global__ void __launch_bounds__(kBlock) k_cg_res_d(Geo g, CgArgs<float> a, const double* xhi,
                                                     const float* x, int all) {
  // runs after every chunk of iterations: with no chain due an update (most
  // chunks) every block returns after one read; otherwise a block visits the
  // site blocks blockIdx.x, + gridDim.x, ...
  if (!all && a.n_active[1] == 0) return;
  for (int blk = blockIdx.x; blk < g.nblocks; blk += gridDim.x) {
    const int c_ = g.blk_chain[blk];
    if (a.grid_mask && !a.grid_mask[c_]) continue;
    const CgChain* cc = a.cgc + c_;
    if (!all && !cc->need_update) continue;
    const ChainInfo ci = g.chains[c_];
    const Site s = site_of(g, ci, c_, blk);
    if (!s.valid) continue;
    auto X = [&](long long m) {
      Sp<double> v = ld_sp(xhi, m);
      if (x) v = v + to_d(ld_sp(x, m));
      return v;
    };
    const long long nxm = at(s, xm1(s), s.t), ntm = at(s, s.x, tm1(s));
    const Lk<double> u = ld_lk(a.U64, s.n);
    const Sp<double> o =
        hop_sum<false, double>(X(at(s, xp1(s), s.t)), X(nxm), X(at(s, s.x, tp1(s))), X(ntm), u.x,
                               ld_lk(a.U64, nxm).x, u.t, ld_lk(a.U64, ntm).t);
    st_sp(a.t64, s.n, (2.0 + ci.m0) * X(s.n) - 0.5 * o);
  }
}

// FP64 residual, step 2: r = b - D^dag t64 and |r|^2.  In update mode
// (!all) also xhi += x, x = 0, r32 = r, and the chain's state advances; in
// report mode only rr_true is written.
__global__ void __launch_bounds__(kBlock) k_cg_res_r(Geo g, CgArgs<float> a, double* xhi,
                                                     int all) {
  if (!all && a.n_active[1] == 0) return;  // as k_cg_res_d
  for (int blk = blockIdx.x; blk < g.nblocks; blk += gridDim.x) {
    const int c_ = g.blk_chain[blk];
    if (a.grid_mask && !a.grid_mask[c_]) continue;
    CgChain* cc = a.cgc + c_;
    if (!all && !cc->need_update) continue;
    const ChainInfo ci = g.chains[c_];
    const Site s = site_of(g, ci, c_, blk);
    double v[1] = {0.0};
    if (s.valid) {
      const long long nxm = at(s, xm1(s), s.t), ntm = at(s, s.x, tm1(s));
      const Lk<double> u = ld_lk(a.U64, s.n);
      const Sp<double> o =
          hop_sum<true, double>(ld_sp(a.t64, at(s, xp1(s), s.t)), ld_sp(a.t64, nxm),
                                ld_sp(a.t64, at(s, s.x, tp1(s))), ld_sp(a.t64, ntm), u.x,
                                ld_lk(a.U64, nxm).x, u.t, ld_lk(a.U64, ntm).t);
      const Sp<double> Ax = (2.0 + ci.m0) * ld_sp(a.t64, s.n) - 0.5 * o;
      const Sp<double> r = ld_sp(a.b, s.n) - Ax;
      v[0] = norm2(r);
      if (!all) {
        st_sp(xhi, s.n, ld_sp_cg(xhi, s.n) + to_d(ld_sp_cg(a.x, s.n)));
        st_sp(a.x, s.n, Sp<float>{{0, 0}, {0, 0}});
        st_sp(a.r, s.n, to_r<float>(r));
      }
    }
    double tot[1];
    if (chain_reduce<1>(v, a.partials, a.counters, g, ci, c_, tot, blk) && threadIdx.x == 0) {
      const double rr = tot[0];
      cc->rr_true = rr;
      if (!all) {
        cc->need_update = 0;
        atomicSub(a.n_active + 1, 1);
        cc->updates += 1;
        cc->alpha_x = 0.0;  // x (with any pending update) is now in xhi
        cc->rmax = rr;
        if (!isfinite(rr)) {
          cc->flags |= 2;
          cc->state = 0;
          atomicSub(a.n_active, 1);
        } else if (rr <= a.tol2 * cc->bb) {
          cc->state = 0;
          atomicSub(a.n_active, 1);
        } else if (cc->iters >= a.maxit) {
          cc->flags |= 1;
          cc->state = 0;
          atomicSub(a.n_active, 1);
        } else {
          cc->beta = rr / cc->rr_prev;
          cc->rr = rr;
          cc->state = 1;
        }
      }
    }
  }
}

// CG kernel timing (sm_profile_enable / sm_profile_read).
struct Profile {
  bool on = false;
  bool ready = false;
  cudaEvent_t e0[2], e1[2], e2[2];  // chunk start, after iterations, after residual
  // deferred solves: one event pair per solve, collected when the caller
  // has synchronised (profile_collect_deferred)
  static constexpr int kPool = 256;
  cudaEvent_t d0[kPool], d1[kPool];
  int nd = 0;
  double iter_ms = 0, res_ms = 0;
  long long batched = 0, site_iters = 0;
};
static Profile g_prof;

// Adds the kernel times of the deferred solves recorded since the last call
// (the stream has been synchronised) and the site-iterations of `iters`.
int profile_collect_deferred(const sm_lattice* L, const int* chain_iters) {
  if (!g_prof.on) return SM_OK;
  for (int i = 0; i < g_prof.nd; ++i) {
    float ms = 0.f;
    SM_CU(cudaEventElapsedTime(&ms, g_prof.d0[i], g_prof.d1[i]));
    g_prof.iter_ms += ms;
  }
  g_prof.nd = 0;
  if (chain_iters)
    for (int c = 0; c < L->nchains; ++c)
      g_prof.site_iters += (long long)chain_iters[c] * L->chains[c].L * L->chains[c].T;
  return SM_OK;
}

static int prof_record(cudaEvent_t* e, int slot, cudaStream_t s) {
  if (!g_prof.on) return SM_OK;
  SM_CU(cudaEventRecord(e[slot], s));
  return SM_OK;
}

// After chunk `slot` is known complete: add its kernel times.
static int prof_collect(int slot, bool residual) {
  if (!g_prof.on) return SM_OK;
  float a = 0.f, b = 0.f;
  SM_CU(cudaEventElapsedTime(&a, g_prof.e0[slot], g_prof.e1[slot]));
  g_prof.iter_ms += a;
  if (residual) {
    SM_CU(cudaEventElapsedTime(&b, g_prof.e1[slot], g_prof.e2[slot]));
    g_prof.res_ms += b;
  }
  return SM_OK;
}

// Chains outside the grid path of a mixed batch start with no pending state.
__global__ void k_cg_reset_masked(CgChain* cgc, const unsigned char* mask, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n && !mask[c]) {
    cgc[c].state = 0;
    cgc[c].need_update = 0;
    cgc[c].alpha_x = 0.0;
  }
}

template <typename R>
static int iterate(Ctx& c, CgArgs<R>& a, int n) {
  if (a.mixed && tiled_cg_applies(c.L))  // large batches: the tiled iteration
    return tiled_cg_iterate(c, (const float*)a.U, (float*)a.r, (float*)a.x, (float*)a.pa,
                            (float*)a.pb, (float*)a.t, a.tol2, a.delta2, a.maxit, n);
  for (int k = 0; k < n; ++k) {
    k_cg_a<R><<<c.grid(), kBlock, 0, c.s>>>(c.g, a);
    int rc = launched(c.st, "cg_a");
    if (rc) return rc;
    k_cg_b<R><<<c.grid(), kBlock, 0, c.s>>>(c.g, a);
    rc = launched(c.st, "cg_b");
    if (rc) return rc;
  }
  return SM_OK;
}

static int residual(Ctx& c, CgArgs<float>& a, double* xhi, const float* x, int all) {
  if (!all && x && tiled_cg_applies(c.L) && c.L->stream_ok) {
    // the fused tiled iteration leaves x += alpha p pending: apply it first
    const int rc = tiled_cg_flush(c, a.x, a.pa, a.pb, a.grid_mask);
    if (rc) return rc;
  }
  const dim3 grid(res_grid(c.L));
  k_cg_res_d<<<grid, kBlock, 0, c.s>>>(c.g, a, xhi, x, all);
  int rc = launched(c.st, "cg_res_d");
  if (rc) return rc;
  k_cg_res_r<<<grid, kBlock, 0, c.s>>>(c.g, a, xhi, all);
  return launched(c.st, "cg_res_r");
}

// The host loop keeps one chunk of iterations in flight: it enqueues chunk
// k+1 before it waits for the active-chain count written after chunk k.
// Iterations enqueued after a chain has converged exit at once.
template <typename R>
static int run(Ctx& c, CgArgs<R>& a, CgArgs<float>& af, int chunk, int maxit, long long* batched,
               long long* updates) {
  int* h = c.L->h_pinned;
  int it = 0, k = 0;
  const int max_chunks = maxit / chunk + 2;
  auto enqueue = [&](int slot) -> int {
    int rc = prof_record(g_prof.e0, slot, c.s);
    if (rc) return rc;
    rc = iterate<R>(c, a, chunk);
    if (rc) return rc;
    if ((rc = prof_record(g_prof.e1, slot, c.s))) return rc;
    it += chunk;
    if (a.mixed) {
      rc = residual(c, af, af.xhi, af.x, 0);
      if (rc) return rc;
    }
    if ((rc = prof_record(g_prof.e2, slot, c.s))) return rc;
    SM_CU(cudaMemcpyAsync(h + slot, a.n_active, sizeof(int), cudaMemcpyDeviceToHost, c.s));
    SM_CU(cudaEventRecord(c.L->ev[slot], c.s));
    return SM_OK;
  };
  int rc = enqueue(0);
  if (rc) return rc;
  for (k = 0; k < max_chunks; ++k) {
    const int slot = k & 1;
    rc = enqueue(slot ^ 1);
    if (rc) return rc;
    SM_CU(cudaEventSynchronize(c.L->ev[slot]));
    if ((rc = prof_collect(slot, a.mixed != 0))) return rc;
    if (h[slot] == 0) break;
  }
  SM_CU(cudaStreamSynchronize(c.s));
  if ((rc = prof_collect((k + 1) & 1, a.mixed != 0))) return rc;
  *batched += it;
  return SM_OK;
}

int cg_solve(Ctx& c, const double* U64, const float* U32, const double* b, double* x,
             const sm_cg_params& cg, int* iters, double* relres, double* dx, bool* have_dx) {
  Range range("cg_solve");
  if (have_dx) *have_dx = false;
  if (!U64 || !b || !x) return fail(SM_ERR_ARG, "cg_solve: NULL field");
  if (!(cg.tol > 0.0) || cg.maxit < 1) return fail(SM_ERR_ARG, "cg_solve: bad tol or maxit");
  const bool mixed = cg.prec == SM_MIXED;
  if (!mixed && cg.prec != SM_F64) return fail(SM_ERR_ARG, "cg_solve: prec must be F64 or MIXED");
  if (mixed && (!U32 || !(cg.delta > 0.0 && cg.delta < 1.0)))
    return fail(SM_ERR_ARG, "cg_solve: MIXED needs U32 and 0 < delta < 1");
  if (b == x) return fail(SM_ERR_ARG, "cg_solve: b and x alias");

  CgArgs<float> af{};
  af.U = U32;
  af.U64 = U64;
  af.b = b;
  af.r = c.w.r32;
  af.x = c.w.x32;
  af.pa = c.w.p32a;
  af.pb = c.w.p32b;
  af.t = c.w.t32;
  af.xhi = x;
  af.t64 = c.w.t;
  af.cgc = c.w.cgc;
  af.partials = c.w.partials;
  af.counters = c.w.counters;
  af.n_active = c.w.n_active;
  af.tol2 = cg.tol * cg.tol;
  af.delta2 = cg.delta * cg.delta;
  af.maxit = cg.maxit;
  af.mixed = mixed ? 1 : 0;

  if (cg.algo < SM_CG_AUTO || cg.algo > SM_CG_CHAIN) return fail(SM_ERR_ARG, "cg_solve: bad algo");
  const bool fits = chain_cg_fits(c.L, cg.prec);
  if (cg.algo == SM_CG_CHAIN && !fits)
    return fail(SM_ERR_ARG, "cg_solve: a chain is too large for the chain-resident solver");
  const bool chain = cg.algo == SM_CG_CHAIN || (cg.algo == SM_CG_AUTO && fits);
  // A batch of both kinds (AUTO, mixed): the chains that fit are solved
  // chain-resident on the side stream while the others iterate grid-wide.
  const bool hybrid = !chain && cg.algo == SM_CG_AUTO && mixed && c.L->nsmall > 0 && !c.deferred;
  // the chain-resident mixed kernels compute D x of the result
  double* dxk = chain && mixed ? dx : nullptr;

  SM_CU(cudaMemsetAsync(c.w.n_active, 0, 2 * sizeof(int), c.s));
  long long batched = 0, updates = 0;
  int rc;
  const int chunk = 8;
  if (chain && c.deferred) {
    // no readback: the chain's flags and iterations accumulate on the device
    const bool timed = g_prof.on && !c.capturing && g_prof.nd < Profile::kPool;
    if (timed) SM_CU(cudaEventRecord(g_prof.d0[g_prof.nd], c.s));
    if ((rc = chain_cg_launch(c, U64, U32, b, x, cg, dxk))) return rc;
    if (timed) SM_CU(cudaEventRecord(g_prof.d1[g_prof.nd++], c.s));
    c.st->cg_solves++;
    if (have_dx) *have_dx = dxk != nullptr;
    return chain_cg_accumulate(c);
  }
  if (chain) {
    if ((rc = prof_record(g_prof.e0, 0, c.s))) return rc;
    if ((rc = chain_cg_launch(c, U64, U32, b, x, cg, dxk))) return rc;
    if (have_dx) *have_dx = dxk != nullptr;
    if ((rc = prof_record(g_prof.e1, 0, c.s))) return rc;
    SM_CU(cudaStreamSynchronize(c.s));
    if ((rc = prof_collect(0, false))) return rc;
  } else if (mixed) {
    if (hybrid) {
      af.grid_mask = c.L->d_grid_mask;
      k_cg_reset_masked<<<(c.L->nchains + 255) / 256, 256, 0, c.s>>>(c.w.cgc, af.grid_mask,
                                                                     c.L->nchains);
      if ((rc = launched(c.st, "cg_reset_masked"))) return rc;
      SM_CU(cudaEventRecord(c.L->ev_fork, c.s));
      SM_CU(cudaStreamWaitEvent(c.L->side, c.L->ev_fork, 0));
      Ctx cs = c;
      cs.s = c.L->side;
      if ((rc = chain_cg_launch_list(cs, U64, U32, b, x, cg))) return rc;
      SM_CU(cudaEventRecord(c.L->ev_join, c.L->side));
    }
    k_cg_init<float><<<c.grid(), kBlock, 0, c.s>>>(c.g, af);
    if ((rc = launched(c.st, "cg_init"))) return rc;
    if ((rc = run<float>(c, af, af, chunk, cg.maxit, &batched, &updates))) return rc;
    if (hybrid) {
      SM_CU(cudaStreamWaitEvent(c.s, c.L->ev_join, 0));
      SM_CU(cudaStreamSynchronize(c.s));
    }
  } else {
    CgArgs<double> ad{};
    ad.U = U64;
    ad.U64 = U64;
    ad.b = b;
    ad.r = c.w.r;
    ad.x = x;
    ad.pa = c.w.p0;
    ad.pb = c.w.p1;
    ad.t = c.w.t;
    ad.xhi = nullptr;
    ad.t64 = c.w.t;
    ad.cgc = c.w.cgc;
    ad.partials = c.w.partials;
    ad.counters = c.w.counters;
    ad.n_active = c.w.n_active;
    ad.tol2 = af.tol2;
    ad.delta2 = af.delta2;
    ad.maxit = cg.maxit;
    ad.mixed = 0;
    k_cg_init<double><<<c.grid(), kBlock, 0, c.s>>>(c.g, ad);
    if ((rc = launched(c.st, "cg_init"))) return rc;
    if ((rc = run<double>(c, ad, af, chunk, cg.maxit, &batched, &updates))) return rc;
    // report the FP64 true residual of the result
    if ((rc = residual(c, af, x, nullptr, 1))) return rc;
  }
  std::vector<CgChain> h(c.L->nchains);
  SM_CU(cudaMemcpyAsync(h.data(), c.w.cgc, sizeof(CgChain) * h.size(), cudaMemcpyDeviceToHost, c.s));
  SM_CU(cudaStreamSynchronize(c.s));
  if (chain) {
    int mx = 0;
    for (const CgChain& ch : h) {
      mx = ch.iters > mx ? ch.iters : mx;
      updates += ch.need_update;
    }
    batched = mx;
  } else if (mixed) {
    // grid-wide chains count their updates; in a hybrid solve the
    // chain-resident ones report theirs in need_update
    for (int i = 0; i < c.L->nchains; ++i)
      updates += (hybrid && !c.L->grid_mask[i]) ? h[i].need_update : h[i].updates;
  }
  c.st->cg_solves++;
  c.st->cg_iterations += batched;
  c.st->reliable_updates += updates;
  if (g_prof.on) {
    g_prof.batched += batched;
    for (int i = 0; i < c.L->nchains; ++i)
      g_prof.site_iters += (long long)h[i].iters * c.L->chains[i].L * c.L->chains[i].T;
  }
  int worst = SM_OK;
  if (!c.strict && c.chain_flags.size() != h.size()) c.chain_flags.assign(h.size(), 0);
  for (int i = 0; i < c.L->nchains; ++i) {
    if (!c.strict) c.chain_flags[i] |= h[i].flags;
    c.st->chain_iterations += h[i].iters;
    if (iters) iters[i] = h[i].iters;
    if (relres) relres[i] = h[i].bb > 0 ? std::sqrt(h[i].rr_true / h[i].bb) : 0.0;
    if (h[i].flags & 2) worst = SM_ERR_NAN;
    else if ((h[i].flags & 1) && worst == SM_OK) worst = SM_ERR_NOT_CONVERGED;
  }
  if (!c.strict) return SM_OK;
  if (worst == SM_ERR_NAN) return fail(SM_ERR_NAN, "cg_solve: breakdown or non-finite residual");
  if (worst == SM_ERR_NOT_CONVERGED) return fail(SM_ERR_NOT_CONVERGED, "cg_solve: maxit reached");
  return SM_OK;
}

}  // namespace sm

using namespace sm;

extern "C" int sm_set_cg_variant(sm_lattice* lat, int variant) {
  if (!lat) return fail(SM_ERR_ARG, "sm_set_cg_variant: lattice is NULL");
  if (variant != -1 && !chain_variant_applies(lat, variant))
    return fail(SM_ERR_ARG, "sm_set_cg_variant: variant %d does not fit these chains", variant);
  lat->cg_variant = variant;
  return SM_OK;
}

extern "C" int sm_autotune_cg(sm_lattice* lat, const double* U64, const float* U32,
                              const double* b, double* x, const sm_cg_params* cg, void* ws,
                              size_t ws_bytes, int* variant, double* ms, void* stream) {
  Ctx c;
  int rc = c.init(lat, ws, ws_bytes, stream, nullptr);
  if (rc) return rc;
  if (!cg || cg->prec != SM_MIXED || !chain_cg_fits(lat, SM_MIXED))
    return fail(SM_ERR_ARG, "sm_autotune_cg: needs SM_MIXED and chains of at most 4096 sites");
  sm_cg_params p = *cg;
  p.algo = SM_CG_CHAIN;
  cudaEvent_t e0, e1;
  SM_CU(cudaEventCreate(&e0));
  SM_CU(cudaEventCreate(&e1));
  int best = 0;
  double best_ms = 1e300;
  for (int v = 0; v < kChainVariants; ++v) {
    if (ms) ms[v] = -1.0;
    if (!chain_variant_applies(lat, v)) continue;
    lat->cg_variant = v;
    double t = 1e300;
    for (int rep = 0; rep < 3; ++rep) {  // the first repetition warms up
      SM_CU(cudaEventRecord(e0, c.s));
      rc = cg_solve(c, U64, U32, b, x, p, nullptr, nullptr);
      if (rc && rc != SM_ERR_NOT_CONVERGED) break;
      SM_CU(cudaEventRecord(e1, c.s));
      SM_CU(cudaEventSynchronize(e1));
      float f = 0.f;
      SM_CU(cudaEventElapsedTime(&f, e0, e1));
      if (rep > 0 && f < t) t = f;
    }
    if (rc && rc != SM_ERR_NOT_CONVERGED) break;
    if (ms) ms[v] = t;
    if (t < best_ms) {
      best_ms = t;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  lat->cg_variant = best;
  if (variant) *variant = best;
  return rc == SM_ERR_NOT_CONVERGED ? SM_OK : rc;
}

extern "C" int sm_profile_enable(int on) {
  if (on && !g_prof.ready) {
    for (int i = 0; i < 2; ++i) {
      SM_CU(cudaEventCreate(&g_prof.e0[i]));
      SM_CU(cudaEventCreate(&g_prof.e1[i]));
      SM_CU(cudaEventCreate(&g_prof.e2[i]));
    }
    for (int i = 0; i < Profile::kPool; ++i) {
      SM_CU(cudaEventCreate(&g_prof.d0[i]));
      SM_CU(cudaEventCreate(&g_prof.d1[i]));
    }
    g_prof.ready = true;
  }
  g_prof.on = on != 0;
  return SM_OK;
}

extern "C" int sm_profile_read(double* iter_ms, double* res_ms, long long* batched_iters,
                               long long* site_iters, int reset) {
  if (iter_ms) *iter_ms = g_prof.iter_ms;
  if (res_ms) *res_ms = g_prof.res_ms;
  if (batched_iters) *batched_iters = g_prof.batched;
  if (site_iters) *site_iters = g_prof.site_iters;
  if (reset) {
    g_prof.iter_ms = g_prof.res_ms = 0;
    g_prof.batched = g_prof.site_iters = 0;
  }
  return SM_OK;
}

extern "C" int sm_cg_solve(const sm_lattice* lat, const double* U64, const float* U32,
                           const double* b, double* x, const sm_cg_params* cg, void* ws,
                           size_t ws_bytes, int* iters, double* relres, void* stream) {
  Ctx c;
  int rc = c.init(lat, ws, ws_bytes, stream, nullptr);
  if (rc) return rc;
  if (!cg) return fail(SM_ERR_ARG, "sm_cg_solve: cg is NULL");
  return cg_solve(c, U64, U32, b, x, *cg, iters, relres);
}
