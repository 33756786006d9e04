// common.cuh -- device helpers shared by the library's translation units:
// complex and two-component spinor arithmetic, batch geometry, and the
// deterministic per-chain reduction used by every FP64 sum.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "schwinger.h"

namespace sm {

// Default bound, in polls of the mbarrier, of a thread block's first wait for
// its TMA box copies (lowered per lattice by sm_set_wait_limit).
constexpr int kTmaSpin = 1 << 22;

constexpr int kBlock = 256;  // threads per site block, one site per thread

// ------------------------------------------------- bounds-checked build ----
//
// Compiled with -DSM_DEBUG (the debug library), every site index of a field
// access (the accessors below) is checked against the site count of the
// call's lattice, and the neighbour and halo indices of the small-lattice
// kernels against their shared-memory extents.  An index out of range is
// counted, the first one recorded with a code for the place it came from,
// and the access goes to index 0 instead: nothing traps, and the host reads
// the record through sm_debug_read.  Each translation unit has its own copy
// of the record (no relocatable device code); the units register their
// set/read functions at load time.  Without SM_DEBUG the checks compile to
// nothing.
#ifdef SM_DEBUG
namespace dbg {
struct Hooks {
  void (*set)(long long sites, cudaStream_t s);  // the extent of site-indexed fields
  void (*take)(unsigned long long* count, long long* first, int* where);  // read and clear
};
int add(const Hooks& h);                            // core.cu
void set_sites(long long sites, cudaStream_t s);    // every unit's extent, on stream s
}  // namespace dbg
static __device__ long long g_dbg_sites = 0x7fffffffffffffffLL;
static __device__ unsigned long long g_dbg_count = 0;
static __device__ long long g_dbg_first = -1;
static __device__ int g_dbg_where = -1;
__device__ __forceinline__ long long dbg_idx(long long i, long long n, int where) {
  if (i >= 0 && i < n) return i;
  if (atomicAdd(&g_dbg_count, 1ull) == 0ull) {
    g_dbg_first = i;
    g_dbg_where = where;
  }
  return 0;
}
static __global__ void k_dbg_set(long long n) { g_dbg_sites = n; }
static void dbg_set(long long n, cudaStream_t s) { k_dbg_set<<<1, 1, 0, s>>>(n); }
static void dbg_take(unsigned long long* count, long long* first, int* where) {
  unsigned long long c = 0;
  long long f = -1;
  int w = -1;
  cudaMemcpyFromSymbol(&c, g_dbg_count, sizeof c);
  cudaMemcpyFromSymbol(&f, g_dbg_first, sizeof f);
  cudaMemcpyFromSymbol(&w, g_dbg_where, sizeof w);
  if (c && *count == 0) {
    *first = f;
    *where = w;
  }
  *count += c;
  const unsigned long long zero = 0;
  const long long none = -1;
  const int nowhere = -1;
  cudaMemcpyToSymbol(g_dbg_count, &zero, sizeof zero);
  cudaMemcpyToSymbol(g_dbg_first, &none, sizeof none);
  cudaMemcpyToSymbol(g_dbg_where, &nowhere, sizeof nowhere);
}
static const int g_dbg_registered = dbg::add(dbg::Hooks{&dbg_set, &dbg_take});
#define SM_IDX(i, n, where) ::sm::dbg_idx((i), (n), (where))
#define SM_SITE(i) ::sm::dbg_idx((i), ::sm::g_dbg_sites, 1)
#else
#define SM_IDX(i, n, where) (i)
#define SM_SITE(i) (i)
#endif

// ------------------------------------------------------------ geometry ----

// One chain of the batch.  Its sites are [off, off + L*T); its site blocks are
// [blk0, blk0 + nblk) of the launch grid of every site kernel.
struct ChainInfo {
  int L, T;
  long long off;
  int blk0, nblk;  // site blocks of the chain
  int tb0, ntb;    // its tiles in the 64 x 16 tile table
  int sb0, nsb;    // its blocks in the fused CG iteration's strip table
  double beta, m0;
};

// Batch geometry as passed to kernels (by value).
struct Geo {
  const ChainInfo* chains;
  const int* blk_chain;  // [nblocks] chain of each site block
  int nblocks;
  int nchains;
};

// A thread's site: global index n, coordinates (x, t) in chain c.
struct Site {
  int c;
  int x, t;
  int L, T;
  long long off;
  long long n;
  bool valid;
};

// Marks a chain of a grid-wide mixed solve as due a reliable update and
// counts it in due[0] (the kernels of the update return at once while that
// count is zero).  Called by the one thread that finishes the chain's
// iteration.
template <typename Chain>
__device__ __forceinline__ void mark_update(Chain* cc, int* due) {
  if (!cc->need_update) {
    cc->need_update = 1;
    atomicAdd(due, 1);
  }
}

// blk: the site block (blockIdx.x, or a block index a looping kernel visits)
__device__ __forceinline__ Site site_of(const Geo& g, const ChainInfo& ci, int c, int blk) {
  Site s;
  s.c = c;
  s.L = ci.L;
  s.T = ci.T;
  s.off = ci.off;
  const int loc = (blk - ci.blk0) * kBlock + threadIdx.x;
  s.valid = loc < ci.L * ci.T;
  const int l = s.valid ? loc : 0;
  s.t = l / ci.L;
  s.x = l - s.t * ci.L;
  s.n = ci.off + l;
  return s;
}
__device__ __forceinline__ Site site_of(const Geo& g, const ChainInfo& ci, int c) {
  return site_of(g, ci, c, blockIdx.x);
}

__device__ __forceinline__ long long at(const Site& s, int x, int t) {
  return s.off + x + (long long)s.L * t;
}
__device__ __forceinline__ int xp1(const Site& s) { return s.x + 1 == s.L ? 0 : s.x + 1; }
__device__ __forceinline__ int xm1(const Site& s) { return s.x == 0 ? s.L - 1 : s.x - 1; }
__device__ __forceinline__ int tp1(const Site& s) { return s.t + 1 == s.T ? 0 : s.t + 1; }
__device__ __forceinline__ int tm1(const Site& s) { return s.t == 0 ? s.T - 1 : s.t - 1; }

// --------------------------------------------------- complex, spinors ----

template <typename R>
struct Cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cx(R re, R im) {
  return Cx<R>{re, im};
}
template <typename R>
__device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) {
  return {a.re - b.re, a.im - b.im};
}
template <typename R>
__device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) {
  return {s * a.re, s * a.im};
}
// conj(a) * b
template <typename R>
__device__ __forceinline__ Cx<R> cmul_conj(Cx<R> a, Cx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename R>
__device__ __forceinline__ Cx<R> conj(Cx<R> a) {
  return {a.re, -a.im};
}
// i * a
template <typename R>
__device__ __forceinline__ Cx<R> mul_i(Cx<R> a) {
  return {-a.im, a.re};
}
template <typename R>
__device__ __forceinline__ R norm2(Cx<R> a) {
  return a.re * a.re + a.im * a.im;
}

template <typename R>
struct Sp {
  Cx<R> a, b;  // spin components 0 and 1
};

template <typename R>
__device__ __forceinline__ Sp<R> operator+(Sp<R> u, Sp<R> v) {
  return {u.a + v.a, u.b + v.b};
}
template <typename R>
__device__ __forceinline__ Sp<R> operator-(Sp<R> u, Sp<R> v) {
  return {u.a - v.a, u.b - v.b};
}
template <typename R>
__device__ __forceinline__ Sp<R> operator*(R s, Sp<R> u) {
  return {s * u.a, s * u.b};
}
template <typename R>
__device__ __forceinline__ R norm2(Sp<R> u) {
  return norm2(u.a) + norm2(u.b);
}
// Re <u, v>
template <typename R>
__device__ __forceinline__ R redot(Sp<R> u, Sp<R> v) {
  return u.a.re * v.a.re + u.a.im * v.a.im + u.b.re * v.b.re + u.b.im * v.b.im;
}

// Spinor fields: [N][2 spins][re, im].  FP32: one 16-byte load per site;
// FP64: two 16-byte loads.
__device__ __forceinline__ Sp<float> ld_sp(const float* p, long long n) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p) + SM_SITE(n));
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ Sp<double> ld_sp(const double* p, long long n) {
  const double2* q = reinterpret_cast<const double2*>(p) + 2 * SM_SITE(n);
  const double2 a = __ldg(q), b = __ldg(q + 1);
  return {{a.x, a.y}, {b.x, b.y}};
}
// loads that bypass L1 (for fields written earlier in the same kernel by
// other blocks never happens; used for read-write fields of the CG)
__device__ __forceinline__ Sp<float> ld_sp_cg(const float* p, long long n) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p) + SM_SITE(n));
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ Sp<double> ld_sp_cg(const double* p, long long n) {
  const double2* q = reinterpret_cast<const double2*>(p) + 2 * SM_SITE(n);
  const double2 a = __ldcg(q), b = __ldcg(q + 1);
  return {{a.x, a.y}, {b.x, b.y}};
}
__device__ __forceinline__ void st_sp(float* p, long long n, Sp<float> v) {
  reinterpret_cast<float4*>(p)[SM_SITE(n)] = make_float4(v.a.re, v.a.im, v.b.re, v.b.im);
}
__device__ __forceinline__ void st_sp(double* p, long long n, Sp<double> v) {
  double2* q = reinterpret_cast<double2*>(p) + 2 * SM_SITE(n);
  q[0] = make_double2(v.a.re, v.a.im);
  q[1] = make_double2(v.b.re, v.b.im);
}

// Links: [N][2 directions][re, im].
template <typename R>
struct Lk {
  Cx<R> x, t;
};
__device__ __forceinline__ Lk<float> ld_lk(const float* U, long long n) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(U) + SM_SITE(n));
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ Lk<double> ld_lk(const double* U, long long n) {
  const double2* q = reinterpret_cast<const double2*>(U) + 2 * SM_SITE(n);
  const double2 a = __ldg(q), b = __ldg(q + 1);
  return {{a.x, a.y}, {b.x, b.y}};
}

// Real link fields (q, p, F, C, v): [N][2].
__device__ __forceinline__ double2 ld_l2(const double* a, long long n) {
  return __ldg(reinterpret_cast<const double2*>(a) + SM_SITE(n));
}
__device__ __forceinline__ double2 ld_l2_cg(const double* a, long long n) {
  return __ldcg(reinterpret_cast<const double2*>(a) + SM_SITE(n));
}
__device__ __forceinline__ void st_l2(double* a, long long n, double2 v) {
  reinterpret_cast<double2*>(a)[SM_SITE(n)] = v;
}

// ------------------------------------------------- Wilson-Dirac hopping ----

// Sum over mu of the four hops of the Wilson-Dirac operator at one site,
// without the factor -1/2:
//   D:     (1 - s_mu) U_mu(n) psi(n+mu) + (1 + s_mu) U_mu(n-mu)^* psi(n-mu)
//   D^dag: (1 + s_mu) U_mu(n) psi(n+mu) + (1 - s_mu) U_mu(n-mu)^* psi(n-mu)
// Each projector 1 -/+ s_mu has rank one:
//   (1 - s1) psi = (a - b)(1, -1)    (1 + s1) psi = (a + b)(1, 1)
//   (1 - s2) psi = (a + ib)(1, -i)   (1 + s2) psi = (a - ib)(1, i)
// so a hop costs one complex multiply by the link.
template <bool DAG, typename R>
__device__ __forceinline__ Sp<R> hop_sum(Sp<R> xp, Sp<R> xm, Sp<R> tp, Sp<R> tm, Cx<R> ux,
                                         Cx<R> uxm, Cx<R> ut, Cx<R> utm) {
  Sp<R> o;
  if (!DAG) {
    const Cx<R> h1 = ux * (xp.a - xp.b);
    const Cx<R> h2 = cmul_conj(uxm, xm.a + xm.b);
    const Cx<R> h3 = ut * (tp.a + mul_i(tp.b));
    const Cx<R> h4 = cmul_conj(utm, tm.a - mul_i(tm.b));
    o.a = (h1 + h2) + (h3 + h4);
    o.b = (h2 - h1) + (mul_i(h4) - mul_i(h3));
  } else {
    const Cx<R> h1 = ux * (xp.a + xp.b);
    const Cx<R> h2 = cmul_conj(uxm, xm.a - xm.b);
    const Cx<R> h3 = ut * (tp.a - mul_i(tp.b));
    const Cx<R> h4 = cmul_conj(utm, tm.a + mul_i(tm.b));
    o.a = (h1 + h2) + (h3 + h4);
    o.b = (h1 - h2) + (mul_i(h3) - mul_i(h4));
  }
  return o;
}

// *p += v in global memory without waiting for the result (a vector
// reduction, performed at L2)
__device__ __forceinline__ void red_add4s(float4* p, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"l"(p), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}

// hop_sum split for walks down a column: hop_tm is the backward t-hop that
// the site above n receives from n, conj(U_t(n)) (1 -/+ s2 projection of f(n)),
// computed while n is the current row; hop_sum_tm adds the other three hops.
template <bool DAG, typename R>
__device__ __forceinline__ Cx<R> hop_tm(Cx<R> ut, Sp<R> f) {
  return cmul_conj(ut, DAG ? f.a + mul_i(f.b) : f.a - mul_i(f.b));
}
template <bool DAG, typename R>
__device__ __forceinline__ Sp<R> hop_sum_tm(Sp<R> xp, Sp<R> xm, Sp<R> tp, Cx<R> ux, Cx<R> uxm,
                                            Cx<R> ut, Cx<R> h4) {
  Sp<R> o;
  if (!DAG) {
    const Cx<R> h1 = ux * (xp.a - xp.b);
    const Cx<R> h2 = cmul_conj(uxm, xm.a + xm.b);
    const Cx<R> h3 = ut * (tp.a + mul_i(tp.b));
    o.a = (h1 + h2) + (h3 + h4);
    o.b = (h2 - h1) + (mul_i(h4) - mul_i(h3));
  } else {
    const Cx<R> h1 = ux * (xp.a + xp.b);
    const Cx<R> h2 = cmul_conj(uxm, xm.a - xm.b);
    const Cx<R> h3 = ut * (tp.a - mul_i(tp.b));
    o.a = (h1 + h2) + (h3 + h4);
    o.b = (h1 - h2) + (mul_i(h3) - mul_i(h4));
  }
  return o;
}

// The bilinears of the fermion force at link (n, mu):
//   A = a(n)^dag (1 - s_mu) U_mu(n) b(n+mu),  B = a(n+mu)^dag (1 + s_mu) U_mu(n)^* b(n)
// (Eq. force_fermion has f = -Im(A - B) with a = chi, b = xi).
template <typename R>
__device__ __forceinline__ void bilinear_x(Sp<R> a, Sp<R> ap, Sp<R> b, Sp<R> bp, Cx<R> u,
                                           Cx<R>& A, Cx<R>& B) {
  A = cmul_conj(a.a - a.b, u * (bp.a - bp.b));
  B = cmul_conj(ap.a + ap.b, cmul_conj(u, b.a + b.b));
}
template <typename R>
__device__ __forceinline__ void bilinear_t(Sp<R> a, Sp<R> ap, Sp<R> b, Sp<R> bp, Cx<R> u,
                                           Cx<R>& A, Cx<R>& B) {
  A = cmul_conj(a.a + mul_i(a.b), u * (bp.a + mul_i(bp.b)));
  B = cmul_conj(ap.a - mul_i(ap.b), cmul_conj(u, b.a - mul_i(b.b)));
}

// ------------------------------------------------------------ reductions --

// Sums NV values over the block in a fixed order; the result is valid in
// thread 0.  Contains __syncthreads: call from all threads of the block.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][kBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][w] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      v[k] = lane < kBlock / 32 ? sh[k][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
  }
}

// Per-chain reduction in two deterministic stages: every block writes its
// partial sums, and the last block of the chain to arrive (ticket counter)
// adds the chain's partials in block order.  Returns true in every thread of
// that last block, with the totals in tot[] of thread 0.  `partials` has
// NV * nblocks entries; `counters` [nchains] must be zero on entry and is
// zero again on exit.
template <int NV>
__device__ __forceinline__ bool chain_reduce(double (&v)[NV], double* partials,
                                             unsigned* counters, const Geo& g,
                                             const ChainInfo& ci, int c, double (&tot)[NV],
                                             int blk = -1) {
  __shared__ bool last;
  if (blk < 0) blk = blockIdx.x;  // the site block whose partials these are
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) __stcg(partials + (size_t)k * g.nblocks + blk, v[k]);
    __threadfence();
    const unsigned prev = atomicAdd(counters + c, 1u);
    last = (prev == (unsigned)ci.nblk - 1u);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = 0.0;
  for (int i = threadIdx.x; i < ci.nblk; i += kBlock)
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] += __ldcg(partials + (size_t)k * g.nblocks + ci.blk0 + i);
  block_sum<NV>(tot);
  if (threadIdx.x == 0) counters[c] = 0u;
  return true;
}

}  // namespace sm
