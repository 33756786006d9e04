// cg_chain.cu -- chain-resident conjugate gradient: one thread block owns one
// chain's entire solve of D^dag D x = b.
//
// For batches of small lattices the grid-wide CG of solver.cu advances all
// chains in lockstep and pays two launches per iteration.  Here every chain
// iterates on its own block with only block barriers, so chains converge
// independently and the whole solve is one launch.  In the FP32 form the links
// U, the search direction p and t = D p live in shared memory (48 bytes per
// site: 192 KB for a 64 x 64 lattice) and the iterate x and residual r in
// registers, so an iteration touches no global memory at all.  The FP64
// reliable update (x_hi += x; r = b - D^dag D x_hi) reads and writes the
// FP64 fields in global memory.  In the FP64 form all fields stay in global
// memory (L2-resident for small chains) and the block still iterates alone.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace sm {

constexpr int kChainThreads = 1024;
// Largest chain volume the shared-memory FP32 form holds (48 B per site).
constexpr int kChainMaxVolume = 4096;

struct ChainCgArgs {
  const ChainInfo* chains;
  const int* list;     // chains handled by this launch, one per block
  const float* U32;
  const double* U64;
  const double* b;
  double* x;           // FP64 solution (global)
  double* t64;         // FP64 scratch [N][2][2]
  double* r64;         // FP64 residual (FP64 form) [N][2][2]
  double* p64;         // FP64 search direction (FP64 form)
  CgChain* cgc;
  double tol2, delta2;
  int maxit;
};

// Sum over the block, returned to every thread (FP64 partials).
__device__ __forceinline__ double cta_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();  // red may still be read from the previous sum
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Block reduction of FP32 per-thread partials: warps add in FP32, the 32
// warp sums are added in FP64 by warp 0, and thread 0 receives the total in
// `fin(total)`, which may update shared scalars.  Ends with a barrier, so
// whatever `fin` wrote is visible to every thread on return.  On GB300 the
// FP64 pipe is a small fraction of the FP32 one: only warp 0 touches it.
template <typename Fin>
__device__ __forceinline__ void cta_reduce(float v, double* red, Fin fin) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) red[w] = (double)v;
  __syncthreads();
  if (w == 0) {
    double s = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) fin(s);
  }
  __syncthreads();
}

// Coordinates and neighbours of local site l of an L x T chain.
struct Nb {
  int l, xp, xm, tp, tm;  // local indices of n, n+x, n-x, n+t, n-t
};
__device__ __forceinline__ Nb neighbours(int l, int L, int T, int lshift) {
  int x, t;
  if (lshift >= 0) {
    x = l & (L - 1);
    t = l >> lshift;
  } else {
    t = l / L;
    x = l - t * L;
  }
  const int row = t * L;
  Nb n;
  // every index is a site of the chain's shared-memory fields (checked in the
  // debug build)
  const int V = L * T;
  n.l = (int)SM_IDX(l, V, 10);
  n.xp = (int)SM_IDX(row + (x + 1 == L ? 0 : x + 1), V, 11);
  n.xm = (int)SM_IDX(row + (x == 0 ? L - 1 : x - 1), V, 12);
  n.tp = (int)SM_IDX((t + 1 == T ? 0 : t + 1) * L + x, V, 13);
  n.tm = (int)SM_IDX((t == 0 ? T - 1 : t - 1) * L + x, V, 14);
  (void)V;
  return n;
}

__device__ __forceinline__ Sp<float> sp_of(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 f4_of(Sp<float> s) {
  return make_float4(s.a.re, s.a.im, s.b.re, s.b.im);
}
__device__ __forceinline__ Sp<double> to_dbl(Sp<float> v) {
  return {{v.a.re, v.a.im}, {v.b.re, v.b.im}};
}
__device__ __forceinline__ Sp<float> to_flt(Sp<double> v) {
  return {{(float)v.a.re, (float)v.a.im}, {(float)v.b.re, (float)v.b.im}};
}

// D (or D^dag) at one site of a field held in shared memory (FP32).
template <bool DAG>
__device__ __forceinline__ Sp<float> dslash_smem(const float4* __restrict__ f,
                                                 const float4* __restrict__ U, const Nb& n,
                                                 float diag) {
  const float4 u = U[n.l];
  const float4 uxm = U[n.xm], utm = U[n.tm];
  const Sp<float> o = hop_sum<DAG, float>(sp_of(f[n.xp]), sp_of(f[n.xm]), sp_of(f[n.tp]),
                                          sp_of(f[n.tm]), {u.x, u.y}, {uxm.x, uxm.y},
                                          {u.z, u.w}, {utm.z, utm.w});
  return diag * sp_of(f[n.l]) - 0.5f * o;
}

// D (or D^dag) at one site of an FP64 field in global memory; `off` is the
// chain's first global site.
template <bool DAG>
__device__ __forceinline__ Sp<double> dslash_glob(const double* __restrict__ f,
                                                  const double* __restrict__ U, long long off,
                                                  const Nb& n, double diag) {
  const Lk<double> u = ld_lk(U, off + n.l);
  const Sp<double> o = hop_sum<DAG, double>(
      ld_sp_cg(f, off + n.xp), ld_sp_cg(f, off + n.xm), ld_sp_cg(f, off + n.tp),
      ld_sp_cg(f, off + n.tm), u.x, ld_lk(U, off + n.xm).x, u.t, ld_lk(U, off + n.tm).t);
  return diag * ld_sp_cg(f, off + n.l) - 0.5 * o;
}

// FP64 true residual of the chain: t64 = D x, r = b - D^dag t64.  Returns
// |r|^2 (to every thread); writes r into r64 if it is not NULL and calls
// put(k, r) for each of the thread's sites.
template <typename Put>
__device__ __forceinline__ double true_residual(const ChainCgArgs& a, const ChainInfo& ci,
                                                int lshift, double* red, Put put) {
  const int V = ci.L * ci.T;
  const double diag = 2.0 + ci.m0;
  for (int l = threadIdx.x; l < V; l += blockDim.x) {
    const Nb n = neighbours(l, ci.L, ci.T, lshift);
    st_sp(a.t64, ci.off + l, dslash_glob<false>(a.x, a.U64, ci.off, n, diag));
  }
  __syncthreads();
  double v = 0.0;
  int k = 0;
  for (int l = threadIdx.x; l < V; l += blockDim.x, ++k) {
    const Nb n = neighbours(l, ci.L, ci.T, lshift);
    const Sp<double> r = ld_sp_cg(a.b, ci.off + l) - dslash_glob<true>(a.t64, a.U64, ci.off, n, diag);
    v += norm2(r);
    put(k, l, r);
  }
  return cta_sum(v, red);
}

// Scalars of a chain-resident solve, owned by thread 0 and broadcast
// through shared memory.
struct ChainScalars {
  double bb, rr, rr_prev, rmax, rr_true;
  float alpha, beta;
  int it, flags, updates;
  int action;  // 0 iterate, 1 reliable update, 2 stop
};

// Mixed precision: FP32 iterations in shared memory and registers, FP64
// reliable updates.  SPT sites per thread (V <= SPT * blockDim.x).
template <int SPT, int NT>
__global__ void __launch_bounds__(NT, 1) k_cg_chain_mixed(ChainCgArgs a) {
  extern __shared__ float4 smem[];
  __shared__ double red[33];
  __shared__ ChainScalars S;
  const int c = a.list[blockIdx.x];
  const ChainInfo ci = a.chains[c];
  const int V = ci.L * ci.T;
  const int lshift = (ci.L & (ci.L - 1)) == 0 ? __ffs(ci.L) - 1 : -1;
  float4* Us = smem;
  float4* ps = smem + V;
  float4* ts = smem + 2 * V;
  const float diag = (float)(2.0 + ci.m0);

  Sp<float> x[SPT], r[SPT];
  double bbl = 0.0;
#pragma unroll
  for (int k = 0; k < SPT; ++k) {
    const int l = threadIdx.x + k * blockDim.x;
    x[k] = {{0.f, 0.f}, {0.f, 0.f}};
    r[k] = x[k];
    if (l < V) {
      Us[l] = __ldg(reinterpret_cast<const float4*>(a.U32) + ci.off + l);
      const Sp<double> bv = ld_sp(a.b, ci.off + l);
      bbl += norm2(bv);
      r[k] = to_flt(bv);
      ps[l] = make_float4(0.f, 0.f, 0.f, 0.f);
      st_sp(a.x, ci.off + l, Sp<double>{{0, 0}, {0, 0}});
    }
  }
  const double bb = cta_sum(bbl, red);
  if (bb == 0.0) {  // x = 0: D x, which the reliable updates otherwise leave in t64
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
      const int l = threadIdx.x + k * blockDim.x;
      if (l < V) st_sp(a.t64, ci.off + l, Sp<double>{{0, 0}, {0, 0}});
    }
  }
  if (threadIdx.x == 0) {
    S.bb = bb;
    S.rr = S.rr_prev = S.rmax = S.rr_true = bb;
    S.beta = 0.f;
    S.it = S.updates = 0;
    S.flags = isfinite(bb) ? 0 : 2;
    S.action = (bb > 0.0 && isfinite(bb)) ? 0 : 2;
  }
  __syncthreads();

  while (S.action != 2) {
    // p <- r + beta p on the thread's own sites
    const float fb = S.beta;
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
      const int l = threadIdx.x + k * blockDim.x;
      if (l < V) ps[l] = f4_of(r[k] + fb * sp_of(ps[l]));
    }
    __syncthreads();
    // t = D p and p^dag A p = |t|^2
    float pap = 0.f;
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
      const int l = threadIdx.x + k * blockDim.x;
      if (l < V) {
        const Sp<float> tv = dslash_smem<false>(ps, Us, neighbours(l, ci.L, ci.T, lshift), diag);
        ts[l] = f4_of(tv);
        pap += norm2(tv);
      }
    }
    cta_reduce(pap, red, [&](double s) {  // its barriers also publish ts
      if (s > 0.0 && isfinite(s)) {
        S.alpha = (float)(S.rr / s);
      } else {
        S.flags |= 2;
        S.action = 2;
      }
    });
    if (S.action == 2) break;
    const float alpha = S.alpha;
    // A p = D^dag t; x += alpha p; r -= alpha A p
    float rn = 0.f;
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
      const int l = threadIdx.x + k * blockDim.x;
      if (l < V) {
        const Sp<float> Ap = dslash_smem<true>(ts, Us, neighbours(l, ci.L, ci.T, lshift), diag);
        x[k] = x[k] + alpha * sp_of(ps[l]);
        r[k] = r[k] - alpha * Ap;
        rn += norm2(r[k]);
      }
    }
    cta_reduce(rn, red, [&](double s) {
      S.rr_prev = S.rr;
      S.rr = s;
      S.beta = (float)(s / S.rr_prev);
      S.it += 1;
      if (!isfinite(s)) {
        S.flags |= 2;
        S.action = 2;
        return;
      }
      S.rmax = fmax(S.rmax, s);
      const bool conv = s <= a.tol2 * S.bb;
      S.action = (conv || s < a.delta2 * S.rmax || S.it >= a.maxit) ? 1 : 0;
    });
    if (S.action == 1) {
      // reliable update: x_hi += x, r = b - A x_hi in FP64
#pragma unroll
      for (int k = 0; k < SPT; ++k) {
        const int l = threadIdx.x + k * blockDim.x;
        if (l < V) {
          st_sp(a.x, ci.off + l, ld_sp_cg(a.x, ci.off + l) + to_dbl(x[k]));
          x[k] = {{0.f, 0.f}, {0.f, 0.f}};
        }
      }
      __syncthreads();
      const double* r64 = a.r64;
      const double rt = true_residual(a, ci, lshift, red, [&](int, int l, const Sp<double>& rv) {
        st_sp(const_cast<double*>(r64), ci.off + l, rv);
      });
#pragma unroll
      for (int k = 0; k < SPT; ++k) {
        const int l = threadIdx.x + k * blockDim.x;
        if (l < V) r[k] = to_flt(ld_sp_cg(a.r64, ci.off + l));
      }
      if (threadIdx.x == 0) {
        S.rr_true = rt;
        S.updates += 1;
        if (!isfinite(rt)) {
          S.flags |= 2;
          S.action = 2;
        } else if (rt <= a.tol2 * S.bb) {
          S.action = 2;
        } else if (S.it >= a.maxit) {
          S.flags |= 1;
          S.action = 2;
        } else {
          S.beta = (float)(rt / S.rr_prev);
          S.rr = rt;
          S.rmax = rt;
          S.action = 0;
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    CgChain* cc = a.cgc + c;
    cc->bb = S.bb;
    cc->rr = S.rr;
    cc->rr_true = S.rr_true;
    cc->iters = S.it;
    cc->flags = S.flags;
    cc->state = 0;
    cc->need_update = S.updates;  // reports the number of reliable updates
  }
}

// FP64 true residual in the column layout (reliable update): t64 = D x_hi,
// then r = b - D^dag t64 on the thread's own strip of R rows of column x,
// walking down the strip with a sliding window (t-neighbours and U_t(n - t)
// from the rows before); x_hi, t64 and U64 are read at L2 (x_hi and t64 were
// written in this kernel by other threads, before a barrier).
struct ColWalk {
  const double* U64;
  long long off;
  int L, T, x, xp, xm, t0;
  double diag;
  __device__ long long row(int t) const {
    return off + (long long)(t < 0 ? t + T : (t >= T ? t - T : t)) * L;
  }
  // (D or D^dag) f at row t0 + j, given f at rows t0 + j - 1 (fm), t0 + j
  // (fc), t0 + j + 1 (fn) and U_t at row t0 + j - 1 (utm); returns U_t of
  // row t0 + j in utm
  template <bool DAG>
  __device__ Sp<double> site(const double* f, int j, const Sp<double>& fm, const Sp<double>& fc,
                             const Sp<double>& fn, Cx<double>& utm) const {
    const long long rw = row(t0 + j);
    const Lk<double> u = ld_lk(U64, rw + x);
    const Sp<double> o = hop_sum<DAG, double>(ld_sp_cg(f, rw + xp), ld_sp_cg(f, rw + xm), fn, fm,
                                              u.x, ld_lk(U64, rw + xm).x, u.t, utm);
    utm = u.t;
    return diag * fc - 0.5 * o;
  }
};

// Double-float numbers for the intermediate reliable updates of the column
// pairs: a value is the unevaluated sum h + l of two floats with |l| below
// an ulp of h (half an ulp after an operation), about 47 significant bits
// (T. J. Dekker, "A floating-point technique for extending the available
// precision", Numer. Math. 18, 1971; the error-free sum of D. E. Knuth,
// TAOCP vol. 2, 4.2.2).
// On GB300 the FP64 pipe runs at 1/64 of the FP32 rate, so a double-float
// D^dag D of a chain costs a fraction of the FP64 one.  The operations are
// written with explicit round-to-nearest intrinsics, which the compiler does
// not fuse or reorder: the error-free transformations depend on it.
struct Df {
  float h, l;
};
// a + b = s + e exactly (Knuth)
__device__ __forceinline__ Df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// a + b = s + e exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ Df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// the sum, with an error of order 2^-47 (|x| + |y|)
__device__ __forceinline__ Df operator+(Df x, Df y) {
  const Df s = df_two_sum(x.h, y.h);
  return df_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ Df operator-(Df x) { return {-x.h, -x.l}; }
__device__ __forceinline__ Df operator-(Df x, Df y) { return x + (-y); }
// the product: x.h y.h exactly as p + e (the fused multiply-add gives the
// rounding error of p), plus the cross terms
__device__ __forceinline__ Df operator*(Df x, Df y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return df_fast_two_sum(p, e);
}
// v truncated to 24 significant bits, as a float, built from v's bits
// (GB300 converts FP64 to FP32 at about half its FP64 add rate; integer
// operations run at the full rate).  Magnitudes below the normal float
// range give 0, above it (and inf, NaN) an infinity.
__device__ __forceinline__ float flt_trunc(double v) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned hi = (unsigned)(u >> 32);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const unsigned m = ((hi & 0xfffffu) << 3) | (unsigned)((u >> 29) & 7u);
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | m);
}
// the FP64 value v as h + l: h is v truncated to a float, v - h is exact in
// FP64 and truncated in turn (h + l within 2^-46 |v| of v; where l would
// fall below the normal float range, within about 1e-38 of it)
__device__ __forceinline__ Df df_of(double v) {
  const float h = flt_trunc(v);
  return {h, flt_trunc(v - (double)h)};
}
__device__ __forceinline__ Cx<Df> df_of(Cx<double> v) { return {df_of(v.re), df_of(v.im)}; }
__device__ __forceinline__ Sp<Df> df_of(const Sp<double>& v) { return {df_of(v.a), df_of(v.b)}; }
__device__ __forceinline__ float flt_of(Df x) { return __fadd_rn(x.h, x.l); }
// half of a spinor (exact)
__device__ __forceinline__ Sp<Df> df_half(const Sp<Df>& v) {
  auto hf = [](Df x) { return Df{0.5f * x.h, 0.5f * x.l}; };
  return {{hf(v.a.re), hf(v.a.im)}, {hf(v.b.re), hf(v.b.im)}};
}
// Double-float fields: 8 floats per site, (h, l) of a.re, a.im, b.re, b.im
// for spinors and of U_x.re, U_x.im, U_t.re, U_t.im for links; they occupy
// the 32 bytes per site of an FP64 spinor field.  Written in the same
// kernel, so read at L2.
__device__ __forceinline__ Sp<Df> ld_spdf(const float* f, long long n) {
  const float4* q = reinterpret_cast<const float4*>(f) + 2 * SM_SITE(n);
  const float4 u = __ldcg(q), v = __ldcg(q + 1);
  return {{{u.x, u.y}, {u.z, u.w}}, {{v.x, v.y}, {v.z, v.w}}};
}
__device__ __forceinline__ void st_spdf(float* f, long long n, const Sp<Df>& s) {
  float4* q = reinterpret_cast<float4*>(f) + 2 * SM_SITE(n);
  q[0] = make_float4(s.a.re.h, s.a.re.l, s.a.im.h, s.a.im.l);
  q[1] = make_float4(s.b.re.h, s.b.re.l, s.b.im.h, s.b.im.l);
}
__device__ __forceinline__ Lk<Df> ld_lkdf(const float* U, long long n) {
  const Sp<Df> v = ld_spdf(U, n);
  return {v.a, v.b};
}
__device__ __forceinline__ Cx<Df> ld_uxdf(const float* U, long long n) {
  const float4 u = __ldcg(reinterpret_cast<const float4*>(U) + 2 * SM_SITE(n));
  return {{u.x, u.y}, {u.z, u.w}};
}

// ColWalk in double-float arithmetic, on double-float copies of x_hi and of
// the links (the same hops in the same order)
struct ColWalkDf {
  const float* U;
  long long off;
  int L, T, x, xp, xm, t0;
  Df diag;
  __device__ long long row(int t) const {
    return off + (long long)(t < 0 ? t + T : (t >= T ? t - T : t)) * L;
  }
  template <bool DAG>
  __device__ Sp<Df> site(const float* f, int j, const Sp<Df>& fm, const Sp<Df>& fc,
                         const Sp<Df>& fn, Cx<Df>& utm) const {
    const long long rw = row(t0 + j);
    const Lk<Df> u = ld_lkdf(U, rw + x);
    const Sp<Df> o = hop_sum<DAG, Df>(ld_spdf(f, rw + xp), ld_spdf(f, rw + xm), fn, fm, u.x,
                                      ld_uxdf(U, rw + xm), u.t, utm);
    utm = u.t;
    return diag * fc - df_half(o);
  }
};

// Column layout for chains whose shape matches the block: thread tid owns
// column x = tid % L and the R consecutive rows t0 .. t0 + R - 1 of row block
// tid / L.  D and D^dag walk down the column with a sliding window, so the
// t-neighbours and the backward t-hop come from registers and only the
// x-neighbours and the links are read from shared memory.  The links are held
// as separate x and t halves, so U_x(n - x) is an 8-byte read, and the
// iterate update x += alpha p waits for the next p update, which reads p
// anyway (the reliable update applies it first).  Every warp finishes the
// block sums itself (FP32, the same order in every warp), so all threads hold
// identical scalars and an iteration needs three barriers.
template <int R, int NT>
__global__ void __launch_bounds__(NT, 1) k_cg_chain_col(ChainCgArgs a) {
  extern __shared__ float4 smem[];
  __shared__ float red[2][NT / 32];
  __shared__ double redd[33];
  const int c = a.list[blockIdx.x];
  const ChainInfo ci = a.chains[c];
  const int L = ci.L, T = ci.T, V = L * T;
  float4* ps = smem;
  float4* ts = smem + V;
  float2* uxs = reinterpret_cast<float2*>(smem + 2 * V);
  float2* uts = uxs + V;
  const float diag = (float)(2.0 + ci.m0);
  const int x = threadIdx.x % L, t0 = (threadIdx.x / L) * R;
  const int xp = x + 1 == L ? 0 : x + 1, xm = x == 0 ? L - 1 : x - 1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  auto site = [&](int t) { return (t < 0 ? t + T : (t >= T ? t - T : t)) * L; };
  auto cx = [](float2 v) { return Cx<float>{v.x, v.y}; };

  // sum of one FP32 value per thread, finished by every warp
  auto bsum = [&](float v, float* buf) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) buf[w] = v;
    __syncthreads();
    float s = lane < NT / 32 ? buf[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
  };

  Sp<float> xv[R], rv[R];
  double bbl = 0.0;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int l = x + (t0 + j) * L;
    const float4 u = __ldg(reinterpret_cast<const float4*>(a.U32) + ci.off + l);
    uxs[l] = make_float2(u.x, u.y);
    uts[l] = make_float2(u.z, u.w);
    const Sp<double> bv = ld_sp(a.b, ci.off + l);
    bbl += norm2(bv);
    rv[j] = to_flt(bv);
    xv[j] = {{0.f, 0.f}, {0.f, 0.f}};
    ps[l] = make_float4(0.f, 0.f, 0.f, 0.f);
    st_sp(a.x, ci.off + l, Sp<double>{{0, 0}, {0, 0}});
  }
  const double bb = cta_sum(bbl, redd);
  if (bb == 0.0)  // x = 0: D x, which the reliable updates otherwise leave in t64
#pragma unroll
    for (int j = 0; j < R; ++j) st_sp(a.t64, ci.off + x + (t0 + j) * L, Sp<double>{{0, 0}, {0, 0}});
  // scalars, identical in every thread; alpha is the last step's, owed to x
  float rr = (float)bb, rr_prev = rr, rmax = rr, beta = 0.f, alpha = 0.f;
  const float tol2bb = (float)(a.tol2 * bb), delta2 = (float)a.delta2;
  double rr_true = bb;
  int it = 0, flags = isfinite(bb) ? 0 : 2, updates = 0;
  bool run = bb > 0.0 && isfinite(bb);

  while (run) {
    // p = r + beta p, and the previous step's x += alpha p
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int l = x + (t0 + j) * L;
      const Sp<float> po = sp_of(ps[l]);
      xv[j] = xv[j] + alpha * po;
      ps[l] = f4_of(rv[j] + beta * po);
    }
    __syncthreads();
    // t = D p down the column
    float pap = 0.f;
    {
      const int rb = site(t0 - 1);
      Cx<float> g = hop_tm<false, float>(cx(uts[x + rb]), sp_of(ps[x + rb]));
      Sp<float> pc = sp_of(ps[x + t0 * L]);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int row = (t0 + j) * L, rn = site(t0 + j + 1);
        const Sp<float> pn = sp_of(ps[x + rn]);
        const Cx<float> ux = cx(uxs[x + row]), ut = cx(uts[x + row]);
        const Sp<float> o = hop_sum_tm<false, float>(sp_of(ps[xp + row]), sp_of(ps[xm + row]), pn,
                                                     ux, cx(uxs[xm + row]), ut, g);
        const Sp<float> tv = diag * pc - 0.5f * o;
        ts[x + row] = f4_of(tv);
        pap += norm2(tv);
        g = hop_tm<false, float>(ut, pc);
        pc = pn;
        asm volatile("" ::: "memory");  // keep the next row's loads after this row
      }
    }
    const float papt = bsum(pap, red[0]);  // its barrier also publishes ts
    if (!(papt > 0.f) || !isfinite(papt)) {
      flags |= 2;
      break;
    }
    alpha = rr / papt;
    // A p = D^dag t down the column; r -= alpha A p
    float rn2 = 0.f;
    {
      const int rb = site(t0 - 1);
      Cx<float> g = hop_tm<true, float>(cx(uts[x + rb]), sp_of(ts[x + rb]));
      Sp<float> tc = sp_of(ts[x + t0 * L]);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int row = (t0 + j) * L, rn = site(t0 + j + 1);
        const Sp<float> tn = sp_of(ts[x + rn]);
        const Cx<float> ux = cx(uxs[x + row]), ut = cx(uts[x + row]);
        const Sp<float> o = hop_sum_tm<true, float>(sp_of(ts[xp + row]), sp_of(ts[xm + row]), tn,
                                                    ux, cx(uxs[xm + row]), ut, g);
        const Sp<float> Ap = diag * tc - 0.5f * o;
        rv[j] = rv[j] - alpha * Ap;
        rn2 += norm2(rv[j]);
        g = hop_tm<true, float>(ut, tc);
        tc = tn;
        asm volatile("" ::: "memory");
      }
    }
    const float rrn = bsum(rn2, red[1]);
    rr_prev = rr;
    rr = rrn;
    beta = rr / rr_prev;
    ++it;
    if (!isfinite(rr)) {
      flags |= 2;
      break;
    }
    rmax = fmaxf(rmax, rr);
    if (rr <= tol2bb || rr < delta2 * rmax || it >= a.maxit) {
      // reliable update: x_hi += x + alpha p, r = b - A x_hi in FP64
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int l = x + (t0 + j) * L;
        const long long n = ci.off + l;
        st_sp(a.x, n, ld_sp_cg(a.x, n) + to_dbl(xv[j] + alpha * sp_of(ps[l])));
        xv[j] = {{0.f, 0.f}, {0.f, 0.f}};
      }
      alpha = 0.f;
      __syncthreads();
      {
        const ColWalk cw{a.U64, ci.off, L, T, x, xp, xm, t0, 2.0 + ci.m0};
        // t64 = D x_hi down the strip
        Sp<double> fm = ld_sp_cg(a.x, cw.row(t0 - 1) + x), fc = ld_sp_cg(a.x, cw.row(t0) + x);
        Cx<double> utm = ld_lk(a.U64, cw.row(t0 - 1) + x).t;
#pragma unroll 1
        for (int j = 0; j < R; ++j) {
          const Sp<double> fn = ld_sp_cg(a.x, cw.row(t0 + j + 1) + x);
          st_sp(a.t64, cw.row(t0 + j) + x, cw.site<false>(a.x, j, fm, fc, fn, utm));
          fm = fc;
          fc = fn;
        }
        __syncthreads();
        // r = b - D^dag t64, into registers (FP32) and |r|^2 (FP64)
        double v = 0.0;
        fm = ld_sp_cg(a.t64, cw.row(t0 - 1) + x);
        fc = ld_sp_cg(a.t64, cw.row(t0) + x);
        utm = ld_lk(a.U64, cw.row(t0 - 1) + x).t;
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const Sp<double> fn = ld_sp_cg(a.t64, cw.row(t0 + j + 1) + x);
          const Sp<double> r =
              ld_sp(a.b, cw.row(t0 + j) + x) - cw.site<true>(a.t64, j, fm, fc, fn, utm);
          v += norm2(r);
          rv[j] = to_flt(r);
          fm = fc;
          fc = fn;
          asm volatile("" ::: "memory");  // one row's loads at a time (registers)
        }
        rr_true = cta_sum(v, redd);
      }
      ++updates;
      if (!isfinite(rr_true)) {
        flags |= 2;
        break;
      }
      if (rr_true <= a.tol2 * bb) break;
      if (it >= a.maxit) {
        flags |= 1;
        break;
      }
      beta = (float)(rr_true / (double)rr_prev);
      rr = (float)rr_true;
      rmax = rr;
    }
    // no barrier here: the next p update reads and writes only the thread's
    // own sites of ps, and the next D stage's writes of ts follow that
    // update's barrier; every read of ts and of neighbouring ps in this
    // iteration precedes the barrier inside the |r|^2 sum above
  }
  if (threadIdx.x == 0) {
    CgChain* cc = a.cgc + c;
    cc->bb = bb;
    cc->rr = rr;
    cc->rr_true = rr_true;
    cc->iters = it;
    cc->flags = flags;
    cc->state = 0;
    cc->need_update = updates;
  }
}

// Cluster helpers for kernels compiled with and without clusters (K = 1:
// the block alone).
template <int K>
__device__ __forceinline__ void ksync() {
  if constexpr (K > 1)
    cooperative_groups::this_cluster().sync();
  else
    __syncthreads();
}
template <int K, typename P>
__device__ __forceinline__ P* kmap(P* p, unsigned r) {
  if constexpr (K > 1)
    return cooperative_groups::this_cluster().map_shared_rank(p, r);
  else
    return p;
}
template <int K>
__device__ __forceinline__ unsigned krank() {
  if constexpr (K > 1)
    return cooperative_groups::this_cluster().block_rank();
  else
    return 0;
}

// Tensor memory (TMEM, 256 KB per SM beside the register file and shared
// memory) as storage for per-thread data a kernel touches once per
// iteration.  A warp reaches the 32 TMEM lanes of its quarter (warp % 4);
// thread i of the warp holds lane 32 (warp % 4) + i, and each tcgen05.ld/st
// below moves 16 consecutive 32-bit columns of that lane to or from 16
// registers.  One warp allocates the columns of the block and frees them
// before the block exits.
// (the load and its wait in one statement: the registers are never read
// before the data has arrived)
__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
// Two 16-column loads and their wait in one statement.
__device__ __forceinline__ void tm_ld16x2(uint32_t ta, uint32_t (&a)[16], uint32_t tb,
                                          uint32_t (&b)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%32];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, "
      "%26, %27, %28, %29, %30, %31}, [%33];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]),
        "=r"(a[7]), "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]),
        "=r"(a[14]), "=r"(a[15]), "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]),
        "=r"(b[5]), "=r"(b[6]), "=r"(b[7]), "=r"(b[8]), "=r"(b[9]), "=r"(b[10]), "=r"(b[11]),
        "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15])
      : "r"(ta), "r"(tb)
      : "memory");
}
// An 8-column load left in flight (tm_wait8 completes it): issued one row
// ahead of its use.  tm_wait8 takes the registers as operands, so nothing
// that reads them can be scheduled before it.
__device__ __forceinline__ void tm_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tm_wait8(uint32_t (&v)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                 "+r"(v[6]), "+r"(v[7])
               :
               : "memory");
}
__device__ __forceinline__ void tm_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};\n" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15])
      : "memory");
}
__device__ __forceinline__ void tm_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}
// A block barrier that orders the tcgen05 operations around it.
__device__ __forceinline__ void tm_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// Allocates `ncols` columns (a power of two, 32 to 512) by warp 0 and
// returns their base address in every thread; ends with a barrier.
__device__ __forceinline__ uint32_t tm_alloc(uint32_t* slot, uint32_t ncols) {
  if ((threadIdx.x >> 5) == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tm_sync();
  return *slot;
}
// Frees the columns (every thread of the block; ends after warp 0 frees).
__device__ __forceinline__ void tm_free(uint32_t base, uint32_t ncols) {
  tm_sync();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(base), "r"(ncols)
                 : "memory");
}

// Column-pair layout for L x T chains (compile-time shape, L * T = 2 R NT K):
// thread tid owns the two columns 2k and 2k + 1 (k = tid % (L/2)) of the R
// rows t0 .. t0 + R - 1 (t0 = (tid / (L/2)) R) of its block's part of the
// chain.  With K > 1 the chain is split over a cluster of K blocks, block
// rank r holding the rows [r T/K, (r+1) T/K); the row below a block's part
// and the row above come from ranks r - 1 and r + 1 (distributed shared
// memory, wrapping with the lattice), and block sums are added across the
// cluster in rank order, so every block takes the same decisions and passes
// the same cluster barriers.  With the shape fixed, every shared-memory
// address of a walk is a per-thread base plus a constant.  Shared memory
// stores every row with its even columns first and its odd columns after
// them, so the x-neighbour between a thread's two sites is its own and the
// two outer ones are the adjacent threads' sites at consecutive addresses (no
// bank conflicts).  The links are held as separate x and t halves, so
// U_x(n - x) is an 8-byte read.  The iterate update x += alpha p waits for
// the next p update, which reads p anyway (the reliable update applies it
// first).  Per site-iteration the 256 x 8 form moves about 162 bytes of
// shared memory, the one-column layout about 202.  Two forms that were
// slower: the FP32 iterate in global memory, updated by vector reductions at
// L2 to free its registers (27 % slower), and the thread's own p kept in
// registers besides shared memory (spills; 24 % slower).
// The float-pair copy of the thread's own links (once per solve), not
// inlined for the same reason as the update walks below.
template <int R, int L>
__device__ __noinline__ void pair_split_links(const double* U64, float* Udf, long long base, int t0,
                                              int k) {
#pragma unroll 1
  for (int i = 0; i < 2 * R; ++i) {
    const long long n = base + (t0 + i / 2) * L + 2 * k + (i & 1);
    const Lk<double> u = ld_lk(U64, n);
    st_spdf(Udf, n, Sp<Df>{df_of(u.x), df_of(u.t)});
  }
}

// The TMEM form's x_hi += x + alpha p at a reliable update (x from tensor
// memory, zeroed after; p from shared memory), with the float-pair copy of
// x_hi when the update is a double-float one.  Four sites' x_hi are loaded
// before any is stored, so the loads overlap.
template <int R, int L>
__device__ __noinline__ void pair_update_x_tm(uint32_t taddr, const float4* ps, float alpha,
                                              double* x, float* xdf, bool fin, long long base,
                                              int t0, int k, int qe, int qo) {
#pragma unroll 1
  for (int ch = 0; ch < 2 * R / 4; ++ch) {
    uint32_t xr[16];
    tm_ld16(taddr + 16 * ch, xr);
    Sp<double> xo[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = 4 * ch + u;
      xo[u] = ld_sp_cg(x, base + (t0 + i / 2) * L + 2 * k + (i & 1));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = 4 * ch + u;
      const int row = (t0 + i / 2) * L;
      const long long n = base + row + 2 * k + (i & 1);
      const Sp<float> xs =
          sp_of(make_float4(__uint_as_float(xr[4 * u]), __uint_as_float(xr[4 * u + 1]),
                            __uint_as_float(xr[4 * u + 2]), __uint_as_float(xr[4 * u + 3]))) +
          alpha * sp_of(ps[row + ((i & 1) ? qo : qe)]);
      const Sp<double> xn = xo[u] + to_dbl(xs);
      st_sp(x, n, xn);
      if (!fin) st_spdf(xdf, n, df_of(xn));
    }
    const uint32_t zero[16] = {};
    tm_st16(taddr + 16 * ch, zero);
  }
  tm_wait_st();
}

// The walks of a reliable update of the column pairs, each a function of
// its own (not inlined: its registers do not weigh on the iteration loop's
// allocation): D x_hi, then r = b - D^dag D x_hi on the thread's columns 2k
// and 2k + 1 from row tg of the chain (t0 of the block's part), r to FP32
// in the thread's own sites of ts; returns the thread's part of |r|^2.
// Double-float form: on the float-pair copies of the links and of x_hi,
// D x_hi to tdf, |r|^2 summed in FP32 (it only sets beta).
template <int R, int L, int T, int K>
__device__ __noinline__ double pair_update_df(const float* Udf, const float* xdf, float* tdf,
                                              const double* b, long long off, double m0, int tg,
                                              int t0, int k, int qe, int qo, float4* ts) {
  const Df dg = df_of(2.0 + m0);
  auto cold = [&](int s) {
    const int xs = 2 * k + s;
    return ColWalkDf{Udf, off, L, T, xs, xs + 1 == L ? 0 : xs + 1, xs == 0 ? L - 1 : xs - 1, tg, dg};
  };
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const ColWalkDf cw = cold(s);
    Sp<Df> fm = ld_spdf(xdf, cw.row(tg - 1) + cw.x), fc = ld_spdf(xdf, cw.row(tg) + cw.x);
    Cx<Df> utm = ld_lkdf(Udf, cw.row(tg - 1) + cw.x).t;
#pragma unroll 1
    for (int j = 0; j < R; ++j) {
      const Sp<Df> fn = ld_spdf(xdf, cw.row(tg + j + 1) + cw.x);
      st_spdf(tdf, cw.row(tg + j) + cw.x, cw.site<false>(xdf, j, fm, fc, fn, utm));
      fm = fc;
      fc = fn;
    }
  }
  ksync<K>();
  float vf = 0.f;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const ColWalkDf cw = cold(s);
    Sp<Df> fm = ld_spdf(tdf, cw.row(tg - 1) + cw.x), fc = ld_spdf(tdf, cw.row(tg) + cw.x);
    Cx<Df> utm = ld_lkdf(Udf, cw.row(tg - 1) + cw.x).t;
#pragma unroll 1
    for (int j = 0; j < R; ++j) {
      const Sp<Df> fn = ld_spdf(tdf, cw.row(tg + j + 1) + cw.x);
      const Sp<Df> rd = df_of(ld_sp(b, cw.row(tg + j) + cw.x)) - cw.site<true>(tdf, j, fm, fc, fn, utm);
      const Sp<float> r{{flt_of(rd.a.re), flt_of(rd.a.im)}, {flt_of(rd.b.re), flt_of(rd.b.im)}};
      vf += norm2(r);
      ts[(t0 + j) * L + (s ? qo : qe)] = f4_of(r);
      fm = fc;
      fc = fn;
    }
  }
  return vf;
}
// FP64 form: t64 = D x_hi (the caller's D x when the solve ends here), |r|^2
// in FP64.
template <int R, int L, int T, int K>
__device__ __noinline__ double pair_update_f64(const double* U64, const double* x, double* t64,
                                               const double* b, long long off, double m0, int tg,
                                               int t0, int k, int qe, int qo, float4* ts) {
  auto col = [&](int s) {
    const int xs = 2 * k + s;
    return ColWalk{U64, off, L, T, xs, xs + 1 == L ? 0 : xs + 1, xs == 0 ? L - 1 : xs - 1, tg,
                   2.0 + m0};
  };
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const ColWalk cw = col(s);
    Sp<double> fm = ld_sp_cg(x, cw.row(tg - 1) + cw.x), fc = ld_sp_cg(x, cw.row(tg) + cw.x);
    Cx<double> utm = ld_lk(U64, cw.row(tg - 1) + cw.x).t;
#pragma unroll 1
    for (int j = 0; j < R; ++j) {
      const Sp<double> fn = ld_sp_cg(x, cw.row(tg + j + 1) + cw.x);
      st_sp(t64, cw.row(tg + j) + cw.x, cw.site<false>(x, j, fm, fc, fn, utm));
      fm = fc;
      fc = fn;
    }
  }
  ksync<K>();
  double v = 0.0;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const ColWalk cw = col(s);
    Sp<double> fm = ld_sp_cg(t64, cw.row(tg - 1) + cw.x), fc = ld_sp_cg(t64, cw.row(tg) + cw.x);
    Cx<double> utm = ld_lk(U64, cw.row(tg - 1) + cw.x).t;
#pragma unroll 1
    for (int j = 0; j < R; ++j) {
      const Sp<double> fn = ld_sp_cg(t64, cw.row(tg + j + 1) + cw.x);
      const Sp<double> r = ld_sp(b, cw.row(tg + j) + cw.x) - cw.site<true>(t64, j, fm, fc, fn, utm);
      v += norm2(r);
      ts[(t0 + j) * L + (s ? qo : qe)] = f4_of(to_flt(r));
      fm = fc;
      fc = fn;
    }
  }
  return v;
}

// Blocks per SM the register budget is sized for: two where a block's part
// of the chain takes at most half an SM's shared memory (clusters of parts
// of 96 KB), else one.
template <int L, int T, int K>
constexpr int pair_min_blocks() {
  return (K > 1 && 48 * L * T / K <= 116 * 1024) ? 2 : 1;
}

// TM (one block, whole warpgroups): the FP32 iterate x, touched once per
// iteration (x += alpha p in the p update, and at a reliable update), lives
// in tensor memory instead of registers (the thread's 2 R sites in 8 R
// columns of its warp's lane quarter), and so do the thread's own links
// (8 R more columns, written once; each walk loads a row's links one row
// ahead of their use), and the thread's own p between iterations (8 R
// more).  The registers x leaves free hold the thread's own p from the p
// update through the D walk and its own t = D p from the D walk through the
// D^dag walk, so neither walk nor the p update reads the thread's own sites
// or own links from shared memory (72 instead of 152 bytes of shared memory
// per site-iteration).  The arithmetic and its order are those of TM = false:
// the results are bitwise the same.  Keeping p in registers across the
// D^dag walk as well spilled 364 bytes and was 11 % slower.
template <int R, int NT, int L, int T, int K, bool TM = false>
__global__ void __launch_bounds__(NT, (pair_min_blocks<L, T, K>())) k_cg_chain_pair(ChainCgArgs a) {
  static_assert(L % 2 == 0 && T % K == 0 && L * T == 2 * R * NT * K,
                "one thread per two columns of R rows");
  static_assert(!TM || (NT % 128 == 0 && R % 2 == 0),
                "TMEM form: whole warpgroups, four sites per 16-column chunk");
  // TMEM form: the thread's 2 R sites of x take 8 R columns, then its own
  // links (U_x, U_t of its two sites, row by row) 8 R more, then its own p
  // 8 R more; the warps of one quarter take consecutive column groups
  constexpr int TMC = 24 * R, TMG = NT / 128;
  constexpr uint32_t TMCOLS = TMC * TMG <= 32 ? 32 : (TMC * TMG <= 64 ? 64 : (TMC * TMG <= 128 ? 128 : (TMC * TMG <= 256 ? 256 : 512)));
  static_assert(NT % 32 == 0 && (T / K) % R == 0 && NT == (L / 2) * (T / K / R),
                "whole warps; the threads tile the part's rows in strips of R");
  constexpr int H = T / K, V = H * L, HL = L / 2;  // rows and sites of a block's part
  extern __shared__ float4 smem[];
  __shared__ __align__(16) float red[2][NT / 32];
  __shared__ double redd[33];
  __shared__ float slot[2];  // this block's part of the two sums of an iteration
  __shared__ float bsum[2];  // the two sums, over the cluster
  __shared__ double slotd;   // this block's part of an FP64 sum
  const unsigned rank = krank<K>();
  const int c = a.list[blockIdx.x / K];
  const ChainInfo ci = a.chains[c];
  const long long base = ci.off + (long long)rank * V;  // first global site of the part
  float4* ps = smem;
  float4* ts = smem + V;
  float2* uxs = reinterpret_cast<float2*>(smem + 2 * V);
  float2* uts = uxs + V;
  // the parts below and above (this block's own with K = 1)
  const unsigned rkb = (rank + K - 1) % K, rka = (rank + 1) % K;
  const float4* psb = kmap<K>(ps, rkb);
  const float4* psa = kmap<K>(ps, rka);
  const float4* tsb = kmap<K>(ts, rkb);
  const float4* tsa = kmap<K>(ts, rka);
  const float2* utsb = kmap<K>(uts, rkb);
  const float diag = (float)(2.0 + ci.m0);
  const int k = threadIdx.x % HL, t0 = (threadIdx.x / HL) * R;
  // positions within a row: the even column 2k, the odd column 2k + 1, the
  // odd column 2k - 1 (x - 1 of the even site), the even column 2k + 2 (x + 1
  // of the odd site)
  const int qe = k, qo = HL + k, qm = HL + (k == 0 ? HL - 1 : k - 1), qp = k + 1 == HL ? 0 : k + 1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ uint32_t tm_slot;
  uint32_t tm_base = 0, taddr = 0;
  if constexpr (TM) {
    tm_base = tm_alloc(&tm_slot, TMCOLS);
    taddr = tm_base + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(TMC * (w >> 2));
  }
  // the rows below and above the thread's strip: offsets in the part that
  // holds them, which is the one below (above) for the strip at the bottom
  // (top) of the part
  const bool bot = t0 == 0, top = t0 + R == H;
  const int rb = bot ? (H - 1) * L : (t0 - 1) * L, ra = top ? 0 : (t0 + R) * L;

  // sum of one FP32 value per thread over the chain, the same in every thread
  auto tsum = [&](float v, int kk) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[kk][w] = v;
    __syncthreads();
    float s;
    if constexpr (NT / 32 == 8) {
      // the eight warp sums read as two 16-byte words and added in the
      // pairing of the butterfly below (whose first two steps add zeros):
      // the same sum, without five dependent shuffles
      const float4 lo = reinterpret_cast<const float4*>(red[kk])[0];
      const float4 hi = reinterpret_cast<const float4*>(red[kk])[1];
      s = ((lo.x + hi.x) + (lo.z + hi.z)) + ((lo.y + hi.y) + (lo.w + hi.w));
    } else {
      s = lane < NT / 32 ? red[kk][lane] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if constexpr (K > 1) {
      // the parts in rank order: lane j of warp 0 reads rank j's part (one
      // distributed-shared-memory load a lane), the warp adds them in rank
      // order and the sum reaches the block through bsum.  Barrier and sum
      // took 0.56 us at K = 8 and 0.63 at 16 this way, 0.66 and 1.32 with
      // every thread reading all K parts (the same additions in the same
      // order: the same result)
      if (threadIdx.x == 0) slot[kk] = s;
      ksync<K>();
      if (w == 0) {
        const float v = lane < K ? kmap<K>(slot, lane)[kk] : 0.f;
        float u = 0.f;
#pragma unroll
        for (int j = 0; j < K; ++j) u += __shfl_sync(0xffffffffu, v, j);
        if (lane == 0) bsum[kk] = u;
      }
      __syncthreads();
      s = bsum[kk];
    }
    return s;
  };
  // FP64 sum over the chain
  auto tsumd = [&](double v) {
    double s = cta_sum(v, redd);
    if constexpr (K > 1) {
      if (threadIdx.x == 0) slotd = s;
      ksync<K>();
      s = 0.0;
#pragma unroll
      for (int j = 0; j < K; ++j) s += *kmap<K>(&slotd, j);
      ksync<K>();  // all have read before slotd is written again
    }
    return s;
  };

  // [2 j] the even site of row t0 + j, [2 j + 1] the odd one.  The TMEM
  // form keeps the thread's own p in registers (pv) and x in TMEM; the
  // other form x in registers (xv) and p in shared memory only.
  Sp<float> rv[2 * R], xv[TM ? 1 : 2 * R], pv[TM ? 2 * R : 1], tv[TM ? 2 * R : 1];
  // double-float copies of the links and of x_hi, and D x_hi of an
  // intermediate reliable update, in the FP64 scratch fields (32 bytes a site)
  float* Udf = reinterpret_cast<float*>(a.p64);
  float* xdf = reinterpret_cast<float*>(a.r64);
  float* tdf = reinterpret_cast<float*>(a.t64);
  double bbl = 0.0;
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) {
    const int row = (t0 + i / 2) * L, l = row + 2 * k + (i & 1), q = row + ((i & 1) ? qo : qe);
    const float4 u = __ldg(reinterpret_cast<const float4*>(a.U32) + base + l);
    // the links times -1/2 (exact): the hop sum then comes out as -o/2, and
    // a site's result diag f - o/2 is one fused multiply-add per component
    uxs[q] = make_float2(-0.5f * u.x, -0.5f * u.y);
    uts[q] = make_float2(-0.5f * u.z, -0.5f * u.w);
    const Sp<double> bv = ld_sp(a.b, base + l);
    bbl += norm2(bv);
    rv[i] = to_flt(bv);
    if constexpr (TM)
      pv[i] = {{0.f, 0.f}, {0.f, 0.f}};
    else
      xv[i] = {{0.f, 0.f}, {0.f, 0.f}};
    ps[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    st_sp(a.x, base + l, Sp<double>{{0, 0}, {0, 0}});
  }
  // the double-float links of the intermediate reliable updates
  pair_split_links<R, L>(a.U64, Udf, base, t0, k);
  if constexpr (TM) {
    const uint32_t zero[16] = {};
#pragma unroll
    for (int ch = 0; ch < 2 * R / 4; ++ch) {
      tm_st16(taddr + 16 * ch, zero);            // x = 0
      tm_st16(taddr + 16 * R + 16 * ch, zero);   // p = 0
    }
    // the links of rows 2 jj and 2 jj + 1, from this thread's own entries of
    // shared memory
#pragma unroll
    for (int jj = 0; jj < R / 2; ++jj) {
      uint32_t lk[16];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = (t0 + 2 * jj + h) * L;
        const float2 ux0 = uxs[row + qe], ut0 = uts[row + qe], ux1 = uxs[row + qo],
                     ut1 = uts[row + qo];
        const float f[8] = {ux0.x, ux0.y, ut0.x, ut0.y, ux1.x, ux1.y, ut1.x, ut1.y};
#pragma unroll
        for (int m = 0; m < 8; ++m) lk[8 * h + m] = __float_as_uint(f[m]);
      }
      tm_st16(taddr + 8 * R + 16 * jj, lk);
    }
    tm_wait_st();
  }
  const double bb = tsumd(bbl);
  if (bb == 0.0)  // x = 0: D x, which the reliable updates otherwise leave in t64
#pragma unroll
    for (int i = 0; i < 2 * R; ++i)
      st_sp(a.t64, base + (t0 + i / 2) * L + 2 * k + (i & 1), Sp<double>{{0, 0}, {0, 0}});
  float rr = (float)bb, rr_prev = rr, rmax = rr, beta = 0.f, alpha = 0.f;
  const float tol2bb = (float)(a.tol2 * bb), delta2 = (float)a.delta2;
  double rr_true = bb;
  int it = 0, flags = isfinite(bb) ? 0 : 2, updates = 0;
  bool run = bb > 0.0 && isfinite(bb);

  // (D or D^dag) f on the thread's two columns, walking down its rows (fb,
  // fa: f of the parts below and above); emit(j, even, odd) receives the two
  // results of row t0 + j
  auto walk = [&](const float4* f, const float4* fb, const float4* fa, auto dag, auto own,
                  auto emit) {
    constexpr bool DAG = decltype(dag)::value;
    // the thread's own sites of f: 0 read from shared memory, 1 pv, 2 tv
    constexpr int OWN = decltype(own)::value;
    auto ownv = [&](int i) -> Sp<float> {
      if constexpr (OWN == 1)
        return pv[i];
      else
        return tv[i];
    };
    auto cx = [](float2 v) { return Cx<float>{v.x, v.y}; };
    const float4* fbr = (bot ? fb : f) + rb;
    const float2* ubr = (bot ? utsb : uts) + rb;
    const float4* far = (top ? fa : f) + ra;
    // the backward t-hops into row t0, then the rows' own hops
    Cx<float> ge = hop_tm<DAG, float>(cx(ubr[qe]), sp_of(fbr[qe]));
    Cx<float> go = hop_tm<DAG, float>(cx(ubr[qo]), sp_of(fbr[qo]));
    // the thread's own links of the current row: from TMEM in the TMEM form,
    // the next row's load in flight while the current one is computed
    uint32_t lk[8], lkn[8];
    if constexpr (TM) {
      tm_ld8(taddr + 8 * R, lk);
      tm_wait8(lk);
    }
    Sp<float> fce, fco;
    if constexpr (OWN != 0) {
      fce = ownv(0);
      fco = ownv(1);
    } else {
      fce = sp_of(f[t0 * L + qe]);
      fco = sp_of(f[t0 * L + qo]);
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int row = (t0 + j) * L;
      Sp<float> fne, fno;  // the row above: the thread's next row, or the strip's row above
      if (j + 1 < R) {      // (an index, not a pointer select: fewer registers)
        if constexpr (OWN != 0) {
          fne = ownv(2 * (j + 1));
          fno = ownv(2 * (j + 1) + 1);
        } else {
          fne = sp_of(f[row + L + qe]);
          fno = sp_of(f[row + L + qo]);
        }
      } else {
        fne = sp_of(far[qe]);
        fno = sp_of(far[qo]);
      }
      Cx<float> uxe, ute, uxo, uto;
      if constexpr (TM) {
        if (j + 1 < R) tm_ld8(taddr + 8 * R + 8 * (j + 1), lkn);
        uxe = {__uint_as_float(lk[0]), __uint_as_float(lk[1])};
        ute = {__uint_as_float(lk[2]), __uint_as_float(lk[3])};
        uxo = {__uint_as_float(lk[4]), __uint_as_float(lk[5])};
        uto = {__uint_as_float(lk[6]), __uint_as_float(lk[7])};
      } else {
        uxe = cx(uxs[row + qe]);
        ute = cx(uts[row + qe]);
        uxo = cx(uxs[row + qo]);
        uto = cx(uts[row + qo]);
      }
      const Sp<float> oe =
          hop_sum_tm<DAG, float>(fco, sp_of(f[row + qm]), fne, uxe, cx(uxs[row + qm]), ute, ge);
      const Sp<float> oo = hop_sum_tm<DAG, float>(sp_of(f[row + qp]), fce, fno, uxo, uxe, uto, go);
      emit(j, diag * fce + oe, diag * fco + oo);
      ge = hop_tm<DAG, float>(ute, fce);
      go = hop_tm<DAG, float>(uto, fco);
      fce = fne;
      fco = fno;
      if constexpr (TM) {
        if (j + 1 < R) {
          tm_wait8(lkn);
#pragma unroll
          for (int m = 0; m < 8; ++m) lk[m] = lkn[m];
        }
      }
      asm volatile("" ::: "memory");  // keep the next row's loads after this row
    }
  };

  while (run) {
    // p = r + beta p, and the previous step's x += alpha p
    if constexpr (TM) {
#pragma unroll
      for (int ch = 0; ch < 2 * R / 4; ++ch) {
        uint32_t xr[16], pr[16];
        tm_ld16x2(taddr + 16 * ch, xr, taddr + 16 * R + 16 * ch, pr);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 4 * ch + u;
          const int row = (t0 + i / 2) * L, q = row + ((i & 1) ? qo : qe);
          const Sp<float> po =
              sp_of(make_float4(__uint_as_float(pr[4 * u]), __uint_as_float(pr[4 * u + 1]),
                                __uint_as_float(pr[4 * u + 2]), __uint_as_float(pr[4 * u + 3])));
          const Sp<float> xs =
              sp_of(make_float4(__uint_as_float(xr[4 * u]), __uint_as_float(xr[4 * u + 1]),
                                __uint_as_float(xr[4 * u + 2]), __uint_as_float(xr[4 * u + 3]))) +
              alpha * po;
          xr[4 * u] = __float_as_uint(xs.a.re);
          xr[4 * u + 1] = __float_as_uint(xs.a.im);
          xr[4 * u + 2] = __float_as_uint(xs.b.re);
          xr[4 * u + 3] = __float_as_uint(xs.b.im);
          pv[i] = rv[i] + beta * po;
          ps[q] = f4_of(pv[i]);
          pr[4 * u] = __float_as_uint(pv[i].a.re);
          pr[4 * u + 1] = __float_as_uint(pv[i].a.im);
          pr[4 * u + 2] = __float_as_uint(pv[i].b.re);
          pr[4 * u + 3] = __float_as_uint(pv[i].b.im);
        }
        tm_st16(taddr + 16 * ch, xr);
        tm_st16(taddr + 16 * R + 16 * ch, pr);
      }
      tm_wait_st();
    } else {
#pragma unroll
      for (int i = 0; i < 2 * R; ++i) {
        const int row = (t0 + i / 2) * L, q = row + ((i & 1) ? qo : qe);
        const Sp<float> po = sp_of(ps[q]);
        xv[i] = xv[i] + alpha * po;
        ps[q] = f4_of(rv[i] + beta * po);
      }
    }
    ksync<K>();  // every part's p (and, the first time, U) is written
    float pap = 0.f;
    walk(ps, psb, psa, std::false_type{}, std::integral_constant<int, TM ? 1 : 0>{},
         [&](int j, const Sp<float>& te, const Sp<float>& to) {
      const int row = (t0 + j) * L;
      ts[row + qe] = f4_of(te);
      ts[row + qo] = f4_of(to);
      if constexpr (TM) {
        tv[2 * j] = te;
        tv[2 * j + 1] = to;
      }
      pap += norm2(te) + norm2(to);
    });
    const float papt = tsum(pap, 0);  // its barrier also publishes ts
    if (!(papt > 0.f) || !isfinite(papt)) {
      flags |= 2;
      break;
    }
    alpha = rr / papt;
    float rn2 = 0.f;
    walk(ts, tsb, tsa, std::true_type{}, std::integral_constant<int, TM ? 2 : 0>{},
         [&](int j, const Sp<float>& ae, const Sp<float>& ao) {
      rv[2 * j] = rv[2 * j] - alpha * ae;
      rv[2 * j + 1] = rv[2 * j + 1] - alpha * ao;
      rn2 += norm2(rv[2 * j]) + norm2(rv[2 * j + 1]);
    });
    const float rrn = tsum(rn2, 1);
    rr_prev = rr;
    rr = rrn;
    beta = rr / rr_prev;
    ++it;
    if (!isfinite(rr)) {
      flags |= 2;
      break;
    }
    rmax = fmaxf(rmax, rr);
    if (rr <= tol2bb || rr < delta2 * rmax || it >= a.maxit) {
      // reliable update: x_hi += x + alpha p, r = b - A x_hi.  An update
      // that may end the solve (the iterated residual at the tolerance, or
      // maxit) computes r in FP64, and the solve ends only on such an update
      // (D x_hi, left in t64, is the caller's D x); the others only restart
      // the FP32 recurrence and compute r in double-float, which is far more
      // precise than that recurrence needs.
      bool fin = rr <= tol2bb || it >= a.maxit;
      if constexpr (TM) {
        pair_update_x_tm<R, L>(taddr, ps, alpha, a.x, xdf, fin, base, t0, k, qe, qo);
      } else {
#pragma unroll
        for (int c4 = 0; c4 < 2 * R; c4 += 4) {
          // four sites' x_hi loaded before any is stored (the loads overlap)
          Sp<double> xo[4];
#pragma unroll
          for (int u = 0; u < 4 && c4 + u < 2 * R; ++u) {
            const int i = c4 + u;
            xo[u] = ld_sp_cg(a.x, base + (t0 + i / 2) * L + 2 * k + (i & 1));
          }
#pragma unroll
          for (int u = 0; u < 4 && c4 + u < 2 * R; ++u) {
            const int i = c4 + u;
            const int row = (t0 + i / 2) * L;
            const long long n = base + row + 2 * k + (i & 1);
            const Sp<float> xs = xv[i] + alpha * sp_of(ps[row + ((i & 1) ? qo : qe)]);
            const Sp<double> xn = xo[u] + to_dbl(xs);
            st_sp(a.x, n, xn);
            if (!fin) st_spdf(xdf, n, df_of(xn));
            xv[i] = {{0.f, 0.f}, {0.f, 0.f}};
          }
        }
      }
      alpha = 0.f;
      for (;;) {
        ksync<K>();
        // the walk down column 2k + s from the strip's first row in the chain
        const int tg = (int)rank * H + t0;
        double v;
        if (!fin)
          v = pair_update_df<R, L, T, K>(Udf, xdf, tdf, a.b, ci.off, ci.m0, tg, t0, k, qe, qo, ts);
        else
          v = pair_update_f64<R, L, T, K>(a.U64, a.x, a.t64, a.b, ci.off, ci.m0, tg, t0, k, qe, qo, ts);
        rr_true = tsumd(v);
#pragma unroll
        for (int i = 0; i < 2 * R; ++i) rv[i] = sp_of(ts[(t0 + i / 2) * L + ((i & 1) ? qo : qe)]);
        ++updates;
        // a double-float update that finds the tolerance met is confirmed by
        // an FP64 one (x_hi unchanged)
        if (fin || !(rr_true <= a.tol2 * bb)) break;
        fin = true;
      }
      if (!isfinite(rr_true)) {
        flags |= 2;
        break;
      }
      if (rr_true <= a.tol2 * bb) break;
      if (it >= a.maxit) {
        flags |= 1;
        break;
      }
      beta = (float)(rr_true / (double)rr_prev);
      rr = (float)rr_true;
      rmax = rr;
    }
    // no barrier here (as in the one-column layout): the next p update
    // touches only the thread's own sites of ps, and every neighbour read of
    // ps and ts in this iteration precedes the barrier of the |r|^2 sum
  }
  if constexpr (K > 1) ksync<K>();  // no block leaves while another may read its shared memory
  if constexpr (TM) tm_free(tm_base, TMCOLS);  // every thread is done with TMEM
  if (threadIdx.x == 0 && rank == 0) {
    CgChain* cc = a.cgc + c;
    cc->bb = bb;
    cc->rr = rr;
    cc->rr_true = rr_true;
    cc->iters = it;
    cc->flags = flags;
    cc->state = 0;
    cc->need_update = updates;
  }
}

// The column layout split over a cluster of K blocks: block rank k owns the
// rows [k T/K, (k+1) T/K) of the chain (U, p, t of those rows in its shared
// memory).  K = 2 at 64 x 64 (96 KB per block, two blocks per SM); K = 4 at
// 128 x 128 (192 KB per block), which keeps such chains chain-resident.  The
// row just below a block's part is read from rank k - 1's shared memory and
// the row just above from rank k + 1's (distributed shared memory; ranks wrap
// around with the lattice), and block sums are combined through it.  Every
// decision is taken on sums that all blocks add in the same order (rank 0's
// part first), so all execute the same sequence of cluster barriers; a final
// barrier keeps a block from exiting while another may still read its shared
// memory.
template <int R, int NT, int K>
__global__ void __launch_bounds__(NT, (K == 2 && NT == 256 ? 2 : 1)) k_cg_chain_cluster(ChainCgArgs a) {
  namespace cgr = cooperative_groups;
  cgr::cluster_group cl = cgr::this_cluster();
  extern __shared__ float4 smem[];
  __shared__ float red[2][NT / 32];
  __shared__ double redd[33];
  __shared__ float slot[2];   // this block's part of the two sums of an iteration
  __shared__ double slotd;    // this block's part of an FP64 sum
  const unsigned rank = cl.block_rank();
  const unsigned rb = (rank + K - 1) % K, ra = (rank + 1) % K;  // ranks below and above
  const int c = a.list[blockIdx.x / K];
  const ChainInfo ci = a.chains[c];
  const int L = ci.L, T = ci.T, H = T / K, HV = H * L;
  const long long base = ci.off + (long long)rank * HV;  // first global site of this part
  float4* Us = smem;
  float4* ps = smem + HV;
  float4* ts = smem + 2 * HV;
  const float4* Ub = cl.map_shared_rank(Us, rb);
  const float4* pb = cl.map_shared_rank(ps, rb);
  const float4* tb = cl.map_shared_rank(ts, rb);
  const float4* Ua = cl.map_shared_rank(Us, ra);
  const float4* pa = cl.map_shared_rank(ps, ra);
  const float4* ta = cl.map_shared_rank(ts, ra);
  const float diag = (float)(2.0 + ci.m0);
  const int x = threadIdx.x % L, t0 = (threadIdx.x / L) * R;  // local rows t0 .. t0 + R - 1
  const int xp = x + 1 == L ? 0 : x + 1, xm = x == 0 ? L - 1 : x - 1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // local row -1 is the last row of the part below, local row H the first
  // row of the part above
  auto at = [&](const float4* own, const float4* below, const float4* above, int lr, int xx) {
    return lr < 0 ? below[(H - 1) * L + xx] : (lr >= H ? above[xx] : own[lr * L + xx]);
  };
  auto ksum = [&](const float* s, int k) {
    float tot = 0.f;
#pragma unroll
    for (int j = 0; j < K; ++j) tot += cl.map_shared_rank(const_cast<float*>(s), j)[k];
    return tot;
  };
  auto ksumd = [&]() {
    double tot = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) tot += *cl.map_shared_rank(&slotd, j);
    return tot;
  };
  // block sum (FP32, finished by every warp), then the cluster sum
  auto csum = [&](float v, int k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[k][w] = v;
    __syncthreads();
    float s = lane < NT / 32 ? red[k][lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) slot[k] = s;
    cl.sync();
    return ksum(slot, k);
  };
  auto csumd = [&](double v) {
    const double s = cta_sum(v, redd);
    if (threadIdx.x == 0) slotd = s;
    cl.sync();
    const double tot = ksumd();
    cl.sync();  // all have read before slotd is written again
    return tot;
  };

  Sp<float> xv[R], rv[R];
  double bbl = 0.0;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int l = x + (t0 + j) * L;
    Us[l] = __ldg(reinterpret_cast<const float4*>(a.U32) + base + l);
    const Sp<double> bv = ld_sp(a.b, base + l);
    bbl += norm2(bv);
    rv[j] = to_flt(bv);
    xv[j] = {{0.f, 0.f}, {0.f, 0.f}};
    ps[l] = make_float4(0.f, 0.f, 0.f, 0.f);
    st_sp(a.x, base + l, Sp<double>{{0, 0}, {0, 0}});
  }
  const double bb = csumd(bbl);
  if (bb == 0.0)  // x = 0: D x, which the reliable updates otherwise leave in t64
#pragma unroll
    for (int j = 0; j < R; ++j) st_sp(a.t64, base + x + (t0 + j) * L, Sp<double>{{0, 0}, {0, 0}});
  float rr = (float)bb, rr_prev = rr, rmax = rr, beta = 0.f;
  const float tol2bb = (float)(a.tol2 * bb), delta2 = (float)a.delta2;
  double rr_true = bb;
  int it = 0, flags = isfinite(bb) ? 0 : 2, updates = 0;
  bool run = bb > 0.0 && isfinite(bb);

  while (run) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int l = x + (t0 + j) * L;
      ps[l] = f4_of(rv[j] + beta * sp_of(ps[l]));
    }
    cl.sync();  // both halves' p (and, first time round, U) are written
    float pap = 0.f;
    {
      Sp<float> pm = sp_of(at(ps, pb, pa, t0 - 1, x)), pc = sp_of(ps[t0 * L + x]);
      float4 um = at(Us, Ub, Ua, t0 - 1, x);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int row = (t0 + j) * L;
        const Sp<float> pn = sp_of(at(ps, pb, pa, t0 + j + 1, x));
        const float4 u = Us[x + row];
        const float4 uxm = Us[xm + row];
        const Sp<float> o = hop_sum<false, float>(sp_of(ps[xp + row]), sp_of(ps[xm + row]), pn,
                                                  pm, {u.x, u.y}, {uxm.x, uxm.y}, {u.z, u.w},
                                                  {um.z, um.w});
        const Sp<float> tv = diag * pc - 0.5f * o;
        ts[x + row] = f4_of(tv);
        pap += norm2(tv);
        pm = pc;
        pc = pn;
        um = u;
      }
    }
    const float papt = csum(pap, 0);  // its cluster barrier also publishes t
    if (!(papt > 0.f) || !isfinite(papt)) {
      flags |= 2;
      break;
    }
    const float alpha = rr / papt;
    float rn2 = 0.f;
    {
      Sp<float> tm = sp_of(at(ts, tb, ta, t0 - 1, x)), tc = sp_of(ts[t0 * L + x]);
      float4 um = at(Us, Ub, Ua, t0 - 1, x);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int row = (t0 + j) * L;
        const Sp<float> tn = sp_of(at(ts, tb, ta, t0 + j + 1, x));
        const float4 u = Us[x + row];
        const float4 uxm = Us[xm + row];
        const Sp<float> o = hop_sum<true, float>(sp_of(ts[xp + row]), sp_of(ts[xm + row]), tn, tm,
                                                 {u.x, u.y}, {uxm.x, uxm.y}, {u.z, u.w},
                                                 {um.z, um.w});
        const Sp<float> Ap = diag * tc - 0.5f * o;
        xv[j] = xv[j] + alpha * sp_of(ps[x + row]);
        rv[j] = rv[j] - alpha * Ap;
        rn2 += norm2(rv[j]);
        tm = tc;
        tc = tn;
        um = u;
      }
    }
    const float rrn = csum(rn2, 1);
    rr_prev = rr;
    rr = rrn;
    beta = rr / rr_prev;
    ++it;
    if (!isfinite(rr)) {
      flags |= 2;
      break;
    }
    rmax = fmaxf(rmax, rr);
    if (rr <= tol2bb || rr < delta2 * rmax || it >= a.maxit) {
      // reliable update on this half: x_hi += x; t64 = D x_hi; r = b - D^dag t64
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const long long n = base + x + (t0 + j) * L;
        st_sp(a.x, n, ld_sp_cg(a.x, n) + to_dbl(xv[j]));
        xv[j] = {{0.f, 0.f}, {0.f, 0.f}};
      }
      cl.sync();
      // t64 = D x_hi, then r = b - D^dag t64, down the thread's strip (its
      // first row in the chain is rank H + t0); rows beyond this block's part
      // are read from global memory like the others, after a cluster barrier
      const ColWalk cw{a.U64, ci.off, L, T, x, xp, xm, (int)rank * H + t0, 2.0 + ci.m0};
      Sp<double> fm = ld_sp_cg(a.x, cw.row(cw.t0 - 1) + x), fc = ld_sp_cg(a.x, cw.row(cw.t0) + x);
      Cx<double> utm = ld_lk(a.U64, cw.row(cw.t0 - 1) + x).t;
#pragma unroll 1
      for (int j = 0; j < R; ++j) {
        const Sp<double> fn = ld_sp_cg(a.x, cw.row(cw.t0 + j + 1) + x);
        st_sp(a.t64, cw.row(cw.t0 + j) + x, cw.site<false>(a.x, j, fm, fc, fn, utm));
        fm = fc;
        fc = fn;
      }
      cl.sync();
      double v = 0.0;
      fm = ld_sp_cg(a.t64, cw.row(cw.t0 - 1) + x);
      fc = ld_sp_cg(a.t64, cw.row(cw.t0) + x);
      utm = ld_lk(a.U64, cw.row(cw.t0 - 1) + x).t;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const Sp<double> fn = ld_sp_cg(a.t64, cw.row(cw.t0 + j + 1) + x);
        const Sp<double> r =
            ld_sp(a.b, cw.row(cw.t0 + j) + x) - cw.site<true>(a.t64, j, fm, fc, fn, utm);
        v += norm2(r);
        rv[j] = to_flt(r);
        fm = fc;
        fc = fn;
        asm volatile("" ::: "memory");  // one row's loads at a time (registers)
      }
      rr_true = csumd(v);
      ++updates;
      if (!isfinite(rr_true)) {
        flags |= 2;
        break;
      }
      if (rr_true <= a.tol2 * bb) break;
      if (it >= a.maxit) {
        flags |= 1;
        break;
      }
      beta = (float)(rr_true / (double)rr_prev);
      rr = (float)rr_true;
      rmax = rr;
    }
  }
  cl.sync();  // no block leaves while another may read its shared memory
  if (threadIdx.x == 0 && rank == 0) {
    CgChain* cc = a.cgc + c;
    cc->bb = bb;
    cc->rr = rr;
    cc->rr_true = rr_true;
    cc->iters = it;
    cc->flags = flags;
    cc->state = 0;
    cc->need_update = updates;
  }
}

// FP64: the same iteration with all fields in global memory (x is the output,
// r64, p64, t64 scratch), one block per chain.
__global__ void __launch_bounds__(kChainThreads, 1) k_cg_chain_f64(ChainCgArgs a) {
  __shared__ double red[33];
  const int c = a.list[blockIdx.x];
  const ChainInfo ci = a.chains[c];
  CgChain* cc = a.cgc + c;
  const int V = ci.L * ci.T;
  const long long off = ci.off;
  const int lshift = (ci.L & (ci.L - 1)) == 0 ? __ffs(ci.L) - 1 : -1;
  const double diag = 2.0 + ci.m0;
  const Sp<double> z = {{0, 0}, {0, 0}};
  double bb = 0.0;
  for (int l = threadIdx.x; l < V; l += blockDim.x) {
    const Sp<double> bv = ld_sp(a.b, off + l);
    bb += norm2(bv);
    st_sp(a.r64, off + l, bv);
    st_sp(a.p64, off + l, z);
    st_sp(a.x, off + l, z);
  }
  bb = cta_sum(bb, red);
  double rr = bb, beta = 0.0;
  int it = 0, flags = 0;
  bool done = !(bb > 0.0) || !isfinite(bb);
  if (!isfinite(bb)) flags |= 2;
  while (!done) {
    for (int l = threadIdx.x; l < V; l += blockDim.x)
      st_sp(a.p64, off + l, ld_sp_cg(a.r64, off + l) + beta * ld_sp_cg(a.p64, off + l));
    __syncthreads();
    double pap = 0.0;
    for (int l = threadIdx.x; l < V; l += blockDim.x) {
      const Sp<double> tv =
          dslash_glob<false>(a.p64, a.U64, off, neighbours(l, ci.L, ci.T, lshift), diag);
      st_sp(a.t64, off + l, tv);
      pap += norm2(tv);
    }
    pap = cta_sum(pap, red);
    if (!(pap > 0.0) || !isfinite(pap)) {
      flags |= 2;
      break;
    }
    const double alpha = rr / pap;
    double rn = 0.0;
    for (int l = threadIdx.x; l < V; l += blockDim.x) {
      const Sp<double> Ap =
          dslash_glob<true>(a.t64, a.U64, off, neighbours(l, ci.L, ci.T, lshift), diag);
      st_sp(a.x, off + l, ld_sp_cg(a.x, off + l) + alpha * ld_sp_cg(a.p64, off + l));
      const Sp<double> rv = ld_sp_cg(a.r64, off + l) - alpha * Ap;
      st_sp(a.r64, off + l, rv);
      rn += norm2(rv);
    }
    rn = cta_sum(rn, red);
    beta = rn / rr;
    rr = rn;
    ++it;
    if (!isfinite(rr)) {
      flags |= 2;
      break;
    }
    if (rr <= a.tol2 * bb) break;
    if (it >= a.maxit) {
      flags |= 1;
      break;
    }
  }
  __syncthreads();
  // report the FP64 true residual of the result
  const double rt = true_residual(a, ci, lshift, red, [](int, int, const Sp<double>&) {});
  if (threadIdx.x == 0) {
    cc->bb = bb;
    cc->rr = rr;
    cc->rr_true = rt;
    cc->iters = it;
    cc->flags = flags;
    cc->state = 0;
    cc->need_update = 0;
  }
}

// Kernel variants of the mixed chain-resident solve: 0 the strided layout
// (any chain up to 4096 sites), 1 the column layout with 512 threads x 8
// rows, 2 the column layout with 256 threads x 16 rows (1 and 2 need every
// chain's shape to match).
bool chain_variant_applies(const sm_lattice* L, int v) {
  if (v == 0) return true;
  if (v < 0 || v > 8) return false;
  if (v >= 5) {
    // column pairs of 64 x 64 chains: 512 threads x 4 rows, 256 x 8, and
    // 2-block clusters of 128 x 8
    for (const ChainInfo& ci : L->chains)
      if (ci.L != 64 || ci.T != 64) return false;
    return true;
  }
  // rows of the chain the column layout covers: 512 x 8, 256 x 16, and for
  // the cluster forms 256 x 8 and 512 x 4 per half
  const int nt = (v == 1 || v == 4) ? 512 : 256, rows = v == 2 ? 16 : (v == 4 ? 4 : 8),
            halves = v >= 3 ? 2 : 1;
  for (const ChainInfo& ci : L->chains)
    if (nt % ci.L != 0 || ci.T != halves * rows * (nt / ci.L)) return false;
  return true;
}


// A chain the 4-block cluster kernel holds: 512 threads per block walk 8-row
// column strips, so L divides 512 and each block owns 8 * 512 / L rows.
bool big_chain_shape(const ChainInfo& ci) {
  return ci.L * ci.T > kChainMaxVolume && 512 % ci.L == 0 && ci.T == 4 * 8 * (512 / ci.L);
}

bool chain_cg_fits(const sm_lattice* L, int prec) {
  int vmax = 0;
  bool all = true;
  for (const ChainInfo& ci : L->chains) {
    vmax = ci.L * ci.T > vmax ? ci.L * ci.T : vmax;
    all = all && (ci.L * ci.T <= kChainMaxVolume || big_chain_shape(ci));
  }
  if (prec == SM_MIXED) return all;
  return vmax <= 4 * kChainMaxVolume;
}

// Launches a K-block-cluster chain kernel: nch chains, K blocks each.
template <int K, typename Kern>
static cudaError_t launch_cluster(Kern kern, int nch, int nt, size_t smem, cudaStream_t s,
                                  const ChainCgArgs& a) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(K * nch));
  cfg.blockDim = dim3((unsigned)nt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = K;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

int chain_cg_prepare(const sm_lattice* L, const sm_cg_params& cg) {
  if (cg.prec != SM_MIXED) return SM_OK;
  // the one-block kernels hold chains of up to kChainMaxVolume sites; larger
  // chains (128 x 128) take the 4-block cluster, whose size is fixed
  int vmax = 1;
  for (const ChainInfo& ci : L->chains)
    if (ci.L * ci.T <= kChainMaxVolume && ci.L * ci.T > vmax) vmax = ci.L * ci.T;
  const int smem = 3 * vmax * (int)sizeof(float4);
  cudaError_t e = cudaFuncSetAttribute(k_cg_chain_cluster<8, 256, 2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem / 2);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_cluster<4, 512, 2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem / 2);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_cluster<8, 512, 4>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 4096 * 16);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_col<8, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_col<16, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_pair<4, 512, 64, 64, 1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_pair<8, 256, 64, 64, 1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_pair<8, 256, 64, 64, 1, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_pair<8, 128, 64, 64, 2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem / 2);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_pair<4, 256, 128, 128, 8, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 2048 * 16);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_pair<2, 64, 16, 16, 1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 256 * 16);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_pair<4, 128, 32, 32, 1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 1024 * 16);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_pair<4, 288, 48, 48, 1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 2304 * 16);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_mixed<1, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_mixed<2, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_chain_mixed<8, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "chain CG attributes: %s", cudaGetErrorString(e));
  return SM_OK;
}

bool chain_cg_selected(const sm_lattice* L, const sm_cg_params& cg) {
  const bool fits = chain_cg_fits(L, cg.prec);
  return cg.algo == SM_CG_CHAIN ? fits : (cg.algo == SM_CG_AUTO && fits);
}

// The chains of `list` in order of decreasing iteration count of their last
// solve (ties by position).  A launch with one block per chain over this
// order starts the longest chains first and gives the SMs that free up the
// shorter ones (blocks are dispatched in index order): consecutive solves on
// similar links take similar iteration counts, so the last wave's idle tail
// shrinks.  The counts are only a guess (any values give a permutation of
// `list`, and a chain's result does not depend on its block).  One block:
// the counts are staged in shared memory (n <= kOrderMax).
constexpr int kOrderMax = 8192;
__global__ void __launch_bounds__(1024) k_chain_order(const CgChain* __restrict__ cgc,
                                                      const int* __restrict__ list,
                                                      int* __restrict__ out, int n) {
  __shared__ int key[kOrderMax];
  for (int j = threadIdx.x; j < n; j += blockDim.x) key[j] = cgc[list[j]].iters;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int ki = key[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) rank += (key[j] > ki) || (key[j] == ki && j < i);
    out[rank] = list[i];
  }
}

// Deferred mode: acc[c] |= flags, acc[nchains + c] += iterations,
// acc[2 nchains + c] += reliable updates.
__global__ void k_cg_accumulate(const CgChain* __restrict__ cgc, int* acc, int nchains) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchains) return;
  acc[c] |= cgc[c].flags;
  acc[nchains + c] += cgc[c].iters;
  acc[2 * nchains + c] += cgc[c].need_update;  // the chain kernels' update count
}

int chain_cg_accumulate(Ctx& c) {
  const int n = c.L->nchains;
  k_cg_accumulate<<<(n + 255) / 256, 256, 0, c.s>>>(c.w.cgc, c.w.acc, n);
  return launched(c.st, "cg_accumulate");
}

int chain_group_kind(const ChainInfo& ci) {
  if (ci.L != ci.T) return 0;
  switch (ci.L) {
    case 16: return 1;
    case 32: return 2;
    case 48: return 3;
    case 64: return 4;
    default: return 0;
  }
}

// Tensor memory of the TMEM forms: 512 columns per block of the one-block
// 64 x 64 kernel (192 KB of shared memory: alone on its SM), 256 per block
// of the 8-block 128 x 128 clusters (96 KB: at most two on an SM); no other
// kernel allocates it, so an allocation never waits.
// Launches the mixed chain-resident solve of one kernel group on stream s,
// the group's chains longest first (by their previous solve).  Column pairs
// per shape (threads x rows per thread): 16 x 16: 64 x 2, 32 x 32: 128 x 4,
// 48 x 48: 288 x 4, 64 x 64: 256 x 8 (each 2 columns wide; at 64 x 64 the
// 256 x 8 form solves faster than 512 x 4 also when its chain has the SM to
// itself, and faster than 4-block clusters of 128 x 4 once the group fills
// the GPU: 2.7 against 4.8 ms for 304 chains, although the clusters take
// 48 chains in 1.1 against 1.5 ms).  Other shapes: the strided kernel.  The
// kernel depends only on the chain's shape, so a chain's result does not
// depend on the rest of its batch.
static int launch_group(Ctx& c, const ChainCgArgs& a0, int g, cudaStream_t s) {
  const sm_lattice* L = c.L;
  ChainCgArgs a = a0;
  const int n = L->group_count[g], kind = L->group_kind[g];
  a.list = L->d_group_list + L->group_begin[g];
  if (kind != 0 && n > 1 && n <= kOrderMax) {
    // the groups order their chains into the end of the order buffer, after
    // the entries of the chains outside the groups (the 128 x 128 clusters,
    // ordered at the same time on another stream, write the start of it)
    int grouped = 0;
    for (int h = 0; h < L->ngroups; ++h) grouped += L->group_count[h];
    int* ord = c.w.order + (L->nchains - grouped) + L->group_begin[g];
    k_chain_order<<<1, 1024, 0, s>>>(c.w.cgc, a.list, ord, n);
    const int rc = launched(c.st, "chain_order");
    if (rc) return rc;
    a.list = ord;
  }
  const size_t smem = (size_t)3 * L->group_vmax[g] * sizeof(float4);
  cudaError_t e = cudaSuccess;
  auto go = [&](auto kern, int nt) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) kern<<<dim3((unsigned)n), dim3(nt), smem, s>>>(a);
  };
  switch (kind) {
    case 1: go(k_cg_chain_pair<2, 64, 16, 16, 1>, 64); break;
    case 2: go(k_cg_chain_pair<4, 128, 32, 32, 1>, 128); break;
    case 3: go(k_cg_chain_pair<4, 288, 48, 48, 1>, 288); break;
    case 4: go(k_cg_chain_pair<8, 256, 64, 64, 1, true>, 256); break;
    default: {
      const int vmax = L->group_vmax[g];
      if (vmax <= 1024)
        go(k_cg_chain_mixed<1, 1024>, 1024);
      else if (vmax <= 2048)
        go(k_cg_chain_mixed<2, 1024>, 1024);
      else
        go(k_cg_chain_mixed<8, 512>, 512);
    }
  }
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "chain CG attribute: %s", cudaGetErrorString(e));
  return launched(c.st, "cg_chain_group");
}

// The chains of at most 4096 sites of a mixed batch (the others untouched):
// one launch per kernel group, the first on c.s, the others on the groups'
// own streams, forked from and joined back into c.s.
int chain_cg_launch_list(Ctx& c, const double* U64, const float* U32, const double* b, double* x,
                         const sm_cg_params& cg, double* dx) {
  const sm_lattice* L = c.L;
  ChainCgArgs a{};
  a.chains = L->d_chains;
  a.U32 = U32;
  a.U64 = U64;
  a.b = b;
  a.x = x;
  a.t64 = dx ? dx : c.w.t;
  a.r64 = c.w.r;
  a.p64 = c.w.p0;
  a.cgc = c.w.cgc;
  a.tol2 = cg.tol * cg.tol;
  a.delta2 = cg.delta * cg.delta;
  a.maxit = cg.maxit;
  if (L->ngroups > 1) {
    cudaError_t e = cudaEventRecord(L->gev_fork, c.s);
    for (int g = 1; g < L->ngroups && e == cudaSuccess; ++g)
      e = cudaStreamWaitEvent(L->gstream[g], L->gev_fork, 0);
    if (e != cudaSuccess) return fail(SM_ERR_CUDA, "chain CG groups fork: %s", cudaGetErrorString(e));
  }
  for (int g = 0; g < L->ngroups; ++g) {
    const int rc = launch_group(c, a, g, g == 0 ? c.s : L->gstream[g]);
    if (rc) return rc;
  }
  for (int g = 1; g < L->ngroups; ++g) {
    cudaError_t e = cudaEventRecord(L->gev_join[g], L->gstream[g]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.s, L->gev_join[g], 0);
    if (e != cudaSuccess) return fail(SM_ERR_CUDA, "chain CG groups join: %s", cudaGetErrorString(e));
  }
  return SM_OK;
}

int chain_cg_launch(Ctx& c, const double* U64, const float* U32, const double* b, double* x,
                    const sm_cg_params& cg, double* dx) {
  const sm_lattice* L = c.L;
  ChainCgArgs a{};
  a.chains = L->d_chains;
  a.list = L->d_chain_list;
  a.U32 = U32;
  a.U64 = U64;
  a.b = b;
  a.x = x;
  a.t64 = dx ? dx : c.w.t;
  a.r64 = c.w.r;
  a.p64 = c.w.p0;
  a.cgc = c.w.cgc;
  a.tol2 = cg.tol * cg.tol;
  a.delta2 = cg.delta * cg.delta;
  a.maxit = cg.maxit;
  const dim3 grid((unsigned)L->nchains), block(kChainThreads);
  (void)block;
  if (cg.prec == SM_MIXED && L->nbig > 0) {
    // small chains on the side stream, clusters for the large ones
    cudaError_t e = cudaEventRecord(L->ev_fork, c.s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(L->side, L->ev_fork, 0);
    if (e != cudaSuccess) return fail(SM_ERR_CUDA, "chain CG fork: %s", cudaGetErrorString(e));
    int rc = SM_OK;
    if (L->nbig < L->nchains) {
      Ctx cs = c;
      cs.s = L->side;
      if ((rc = chain_cg_launch_list(cs, U64, U32, b, x, cg, dx))) return rc;
    }
    ChainCgArgs ab = a;
    ab.list = L->d_big_list;
    bool sq128 = true;  // all large chains 128 x 128: the column-pair form
    for (const ChainInfo& ci : L->chains)
      if (ci.L * ci.T > kChainMaxVolume) sq128 = sq128 && ci.L == 128 && ci.T == 128;
    if (sq128 && L->nbig <= kOrderMax) {
      // the clusters longest first, as for the one-block column pairs
      k_chain_order<<<1, 1024, 0, c.s>>>(c.w.cgc, L->d_big_list, c.w.order, L->nbig);
      if ((rc = launched(c.st, "chain_order"))) return rc;
      ab.list = c.w.order;
    }
    if (sq128)
      e = launch_cluster<8>(k_cg_chain_pair<4, 256, 128, 128, 8, true>, L->nbig, 256,
                            (size_t)3 * 2048 * 16, c.s, ab);
    else
      e = launch_cluster<4>(k_cg_chain_cluster<8, 512, 4>, L->nbig, 512, (size_t)3 * 4096 * 16,
                            c.s, ab);
    if (e != cudaSuccess) return fail(SM_ERR_CUDA, "chain CG (clusters): %s", cudaGetErrorString(e));
    if ((rc = launched(c.st, "cg_chain_cluster4"))) return rc;
    e = cudaEventRecord(L->ev_join, L->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.s, L->ev_join, 0);
    if (e != cudaSuccess) return fail(SM_ERR_CUDA, "chain CG join: %s", cudaGetErrorString(e));
    return SM_OK;
  }
  if (cg.prec == SM_MIXED) {
    int vmax = 0;
    for (const ChainInfo& ci : L->chains) vmax = ci.L * ci.T > vmax ? ci.L * ci.T : vmax;
    const size_t smem = (size_t)3 * vmax * sizeof(float4);
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern, int nt) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) kern<<<grid, dim3(nt), smem, c.s>>>(a);
    };
    int v = L->cg_variant;
    if (v < 0 && L->ngroups > 0) {
      // not pinned: one launch per kernel group
      const int rc = chain_cg_launch_list(c, U64, U32, b, x, cg, dx);
      if (rc) return rc;
      return SM_OK;
    }
    if (v < 0 || !chain_variant_applies(L, v)) v = 0;
    if (v == 3) {
      e = launch_cluster<2>(k_cg_chain_cluster<8, 256, 2>, L->nchains, 256, smem / 2, c.s, a);
    } else if (v == 4) {
      e = launch_cluster<2>(k_cg_chain_cluster<4, 512, 2>, L->nchains, 512, smem / 2, c.s, a);
    } else if (v == 1) {
      go(k_cg_chain_col<8, 512>, 512);
    } else if (v == 2) {
      go(k_cg_chain_col<16, 256>, 256);
    } else if (v == 5 || v == 6 || v == 8) {
      // one block per chain, the chains longest first (k_chain_order)
      const int n = L->nchains;
      ChainCgArgs ao = a;
      if (n <= kOrderMax) {
        k_chain_order<<<1, 1024, 0, c.s>>>(c.w.cgc, L->d_chain_list, c.w.order, n);
        const int rc = launched(c.st, "chain_order");
        if (rc) return rc;
        ao.list = c.w.order;
      }
      auto kern = v == 5   ? k_cg_chain_pair<4, 512, 64, 64, 1>
                  : v == 6 ? k_cg_chain_pair<8, 256, 64, 64, 1>
                           : k_cg_chain_pair<8, 256, 64, 64, 1, true>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) kern<<<grid, dim3(v == 5 ? 512 : 256), smem, c.s>>>(ao);
    } else if (v == 7) {
      e = launch_cluster<2>(k_cg_chain_pair<8, 128, 64, 64, 2>, L->nchains, 128, smem / 2, c.s, a);
    } else if (vmax <= 1024) {
      // x and r of every site live in registers: 8 floats per site, so the
      // largest chains use 512 threads with 8 sites each (up to 128
      // registers per thread) rather than 1024 threads with 4 (64: spills).
      go(k_cg_chain_mixed<1, 1024>, 1024);
    } else if (vmax <= 2048) {
      go(k_cg_chain_mixed<2, 1024>, 1024);
    } else {
      go(k_cg_chain_mixed<8, 512>, 512);
    }
    if (e != cudaSuccess) return fail(SM_ERR_CUDA, "chain CG attribute: %s", cudaGetErrorString(e));
    return launched(c.st, "cg_chain_mixed");
  }
  k_cg_chain_f64<<<grid, dim3(kChainThreads), 0, c.s>>>(a);
  return launched(c.st, "cg_chain_f64");
}

}  // namespace sm
