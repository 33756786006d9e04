// core.cu -- lattice objects, workspace, error reporting, and the site
// kernels of the Schwinger-model hot path: links, the Wilson-Dirac operator,
// the gauge and fermion forces, the pieces of the exact force-gradient term,
// link-field linear combinations and the per-chain energy sums.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sm {

static thread_local char g_err[512] = "no error";
static std::atomic<long long> g_launches{0};

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int launched(sm_stats* st, const char* what) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (st) st->kernel_launches++;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "launch of %s: %s", what, cudaGetErrorString(e));
  return SM_OK;
}

#define SM_CU(call)                                                                      \
  do {                                                                                   \
    const cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return fail(SM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------- workspace ----

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

size_t Ws::bytes(const sm_lattice* L) {
  const size_t N = (size_t)L->N, nb = (size_t)L->nblocks, nc = (size_t)L->nchains;
  size_t b = 0;
  b += 12 * align256(N * 32);          // FP64 spinors
  b += 5 * align256(N * 16);           // FP32 spinors
  b += 2 * align256(N * 32);           // U64, U64s
  b += 2 * align256(N * 16);           // U32, U32s
  b += 7 * align256(N * 16);           // link fields
  b += align256(N * sizeof(double));   // plaquette sines
  b += align256(4 * nb * sizeof(double));
  b += align256(nc * sizeof(unsigned));
  b += align256(nc * sizeof(CgChain));
  b += align256(8 * nc * sizeof(double));
  b += align256(nc * sizeof(int));
  b += align256(3 * nc * sizeof(int));
  b += align256(2 * sizeof(int));
  b += align256(nc * sizeof(int));
  if (L->heavy) b += 2 * align256(N * 32);  // phi_h, psi
  return b;
}

int Ws::carve(const sm_lattice* L, void* ws, size_t nbytes) {
  if (!ws) return fail(SM_ERR_ARG, "workspace is NULL");
  if (((uintptr_t)ws & 255) != 0) return fail(SM_ERR_ARG, "workspace not 256-byte aligned");
  if (nbytes < bytes(L))
    return fail(SM_ERR_ARG, "workspace too small: %zu < %zu bytes", nbytes, bytes(L));
  const size_t N = (size_t)L->N, nb = (size_t)L->nblocks, nc = (size_t)L->nchains;
  char* p = static_cast<char*>(ws);
  auto take = [&](size_t b) {
    char* r = p;
    p += align256(b);
    return r;
  };
  double** d64[] = {&r, &t, &p0, &p1, &xi, &chi, &s1, &s2, &z1, &z2, &phi, &b};
  for (double** d : d64) *d = reinterpret_cast<double*>(take(N * 32));
  float** f32[] = {&r32, &x32, &p32a, &p32b, &t32};
  for (float** f : f32) *f = reinterpret_cast<float*>(take(N * 16));
  U64 = reinterpret_cast<double*>(take(N * 32));
  U64s = reinterpret_cast<double*>(take(N * 32));
  U32 = reinterpret_cast<float*>(take(N * 16));
  U32s = reinterpret_cast<float*>(take(N * 16));
  double** lf[] = {&F, &C, &F2, &qs, &qsave, &pw, &v};
  for (double** d : lf) *d = reinterpret_cast<double*>(take(N * 16));
  sinp = reinterpret_cast<double*>(take(N * sizeof(double)));
  partials = reinterpret_cast<double*>(take(4 * nb * sizeof(double)));
  counters = reinterpret_cast<unsigned*>(take(nc * sizeof(unsigned)));
  cgc = reinterpret_cast<CgChain*>(take(nc * sizeof(CgChain)));
  out = reinterpret_cast<double*>(take(8 * nc * sizeof(double)));
  flags = reinterpret_cast<int*>(take(nc * sizeof(int)));
  acc = reinterpret_cast<int*>(take(3 * nc * sizeof(int)));
  n_active = reinterpret_cast<int*>(take(2 * sizeof(int)));
  order = reinterpret_cast<int*>(take(nc * sizeof(int)));
  phi_h = psi = nullptr;
  if (L->heavy) {
    phi_h = reinterpret_cast<double*>(take(N * 32));
    psi = reinterpret_cast<double*>(take(N * 32));
  }
  h_n_active = L->h_pinned;
  return SM_OK;
}

#ifdef SM_DEBUG
namespace dbg {
static std::vector<Hooks>& hooks() {
  static std::vector<Hooks> h;  // constructed on first use (units register at load time)
  return h;
}
int add(const Hooks& h) {
  hooks().push_back(h);
  return (int)hooks().size();
}
void set_sites(long long sites, cudaStream_t s) {
  for (const Hooks& h : hooks()) h.set(sites, s);
}
}  // namespace dbg
#endif

int Ctx::init(const sm_lattice* lat, void* ws, size_t nbytes, void* stream, sm_stats* stats,
               bool ws_required) {
  if (!lat) return fail(SM_ERR_ARG, "lattice is NULL");
  if (ws_required && !ws) return fail(SM_ERR_ARG, "workspace is NULL");
#ifdef SM_DEBUG
  dbg::set_sites(lat->N, static_cast<cudaStream_t>(stream));
#endif
  L = lat;
  g.chains = lat->d_chains;
  g.blk_chain = lat->d_blk_chain;
  g.nblocks = lat->nblocks;
  g.nchains = lat->nchains;
  s = static_cast<cudaStream_t>(stream);
  memset(&local, 0, sizeof local);
  st = stats ? stats : &local;
  memset(st, 0, sizeof *st);
  if (ws) {
    const int rc = w.carve(lat, ws, nbytes);
    if (rc) return rc;
    return zero_counters();
  }
  memset(&w, 0, sizeof w);
  return SM_OK;
}

int Ctx::zero_counters() {
  SM_CU(cudaMemsetAsync(w.counters, 0, sizeof(unsigned) * (size_t)L->nchains, s));
  return SM_OK;
}

int Ctx::sync() {
  SM_CU(cudaStreamSynchronize(s));
  return SM_OK;
}

int Ctx::read_n_active(int* n) {
  SM_CU(cudaMemcpyAsync(w.h_n_active, w.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
  SM_CU(cudaStreamSynchronize(s));
  *n = *w.h_n_active;
  return SM_OK;
}

// ------------------------------------------------------------- kernels ----

#define SITE_PROLOGUE                                 \
  const int c_ = g.blk_chain[blockIdx.x];             \
  const ChainInfo ci = g.chains[c_];                  \
  const Site s = site_of(g, ci, c_);

// U_mu(n) = exp(i q_mu(n)); t-links on the last time slice carry the
// antiperiodic fermion sign.
__global__ void __launch_bounds__(kBlock) k_links(Geo g, const double* __restrict__ q,
                                                  double* __restrict__ U64,
                                                  float* __restrict__ U32) {
  SITE_PROLOGUE
  if (!s.valid) return;
  const double2 a = ld_l2(q, s.n);
  double sx, cx, st, ct;
  sincos(a.x, &sx, &cx);
  sincos(a.y, &st, &ct);
  if (s.t == s.T - 1) {
    st = -st;
    ct = -ct;
  }
  if (U64) {
    double2* u = reinterpret_cast<double2*>(U64) + 2 * s.n;
    u[0] = make_double2(cx, sx);
    u[1] = make_double2(ct, st);
  }
  if (U32) reinterpret_cast<float4*>(U32)[s.n] = make_float4((float)cx, (float)sx, (float)ct, (float)st);
}

template <typename R>
__device__ __forceinline__ Cx<R> link_x(const R* U, long long n) {
  return ld_lk(U, n).x;
}
template <typename R>
__device__ __forceinline__ Cx<R> link_t(const R* U, long long n) {
  return ld_lk(U, n).t;
}

// out = D in (or D^dag in) + add_scale * add.
template <typename R, bool DAG>
__global__ void __launch_bounds__(kBlock) k_dslash(Geo g, const R* __restrict__ U,
                                                   const R* __restrict__ in, R* __restrict__ out,
                                                   const R* __restrict__ add, R add_scale) {
  SITE_PROLOGUE
  if (!s.valid) return;
  const int xp = xp1(s), xm = xm1(s), tp = tp1(s), tm = tm1(s);
  const Lk<R> u = ld_lk(U, s.n);
  const Sp<R> o = hop_sum<DAG, R>(ld_sp(in, at(s, xp, s.t)), ld_sp(in, at(s, xm, s.t)),
                                  ld_sp(in, at(s, s.x, tp)), ld_sp(in, at(s, s.x, tm)), u.x,
                                  link_x(U, at(s, xm, s.t)), u.t, link_t(U, at(s, s.x, tm)));
  Sp<R> r = (R)(2.0 + ci.m0) * ld_sp(in, s.n) - (R)0.5 * o;
  if (add) r = r + add_scale * ld_sp(add, s.n);
  st_sp(out, s.n, r);
}

// Plaquette angle th(m) = q_x(m) + q_t(m+x) - q_x(m+t) - q_t(m) from the
// angles at m, m+x, m+t.
__device__ __forceinline__ double plaq_angle(double2 qm, double2 qmx, double2 qmt) {
  return qm.x + qmx.y - qmt.x - qm.y;
}

// The seven sites a gauge-force or gauge-Hessian stencil reads.
struct GaugeNb {
  long long n, nx, nt, nmt, nxmt, nmx, nmxt;  // n, n+x, n+t, n-t, n+x-t, n-x, n-x+t
};
__device__ __forceinline__ GaugeNb gauge_nb(const Site& s) {
  const int xp = xp1(s), xm = xm1(s), tp = tp1(s), tm = tm1(s);
  return {s.n, at(s, xp, s.t), at(s, s.x, tp), at(s, s.x, tm), at(s, xp, tm), at(s, xm, s.t),
          at(s, xm, tp)};
}

// The same in one pass, three sines per site (for callers without a
// workspace, which has the scratch field of the two-pass form).
__global__ void __launch_bounds__(kBlock) k_gauge_kick_direct(Geo g, const double* __restrict__ q,
                                                              double* __restrict__ Fout) {
  SITE_PROLOGUE
  if (!s.valid) return;
  const GaugeNb b = gauge_nb(s);
  const double2 q0 = ld_l2(q, b.n), qx = ld_l2(q, b.nx), qt = ld_l2(q, b.nt);
  const double2 qmt = ld_l2(q, b.nmt), qxmt = ld_l2(q, b.nxmt);
  const double2 qmx = ld_l2(q, b.nmx), qmxt = ld_l2(q, b.nmxt);
  const double s0 = sin(plaq_angle(q0, qx, qt));
  const double s_mt = sin(plaq_angle(qmt, qxmt, q0));
  const double s_mx = sin(plaq_angle(qmx, q0, qmxt));
  st_l2(Fout, s.n, make_double2(ci.beta * (s0 - s_mt), ci.beta * (s_mx - s0)));
}

// sin th(n) of the plaquette at every site (Eq. plaquette), one sine per
// plaquette: the gauge kick below reads it at n, n - t and n - x, so the
// FP64 sine (the kernel's cost on GB300's FP64 pipe) is taken once, not
// three times, per plaquette.
__global__ void __launch_bounds__(kBlock) k_plaq_sin(Geo g, const double* __restrict__ q,
                                                     double* __restrict__ S) {
  SITE_PROLOGUE
  if (!s.valid) return;
  const long long nx = at(s, xp1(s), s.t), nt = at(s, s.x, tp1(s));
  S[s.n] = sin(plaq_angle(ld_l2(q, s.n), ld_l2(q, nx), ld_l2(q, nt)));
}

// p -= eps F_G and/or Fout (=, or += if acc) F_G, with F_G = beta g of
// Eq. force_gauge: F(n,x) = beta [sin th(n) - sin th(n-t)],
//                  F(n,t) = beta [sin th(n-x) - sin th(n)],
// from S = sin th of k_plaq_sin.
__global__ void __launch_bounds__(kBlock) k_gauge_kick(Geo g, const double* __restrict__ S,
                                                       double* __restrict__ p, double eps,
                                                       double* __restrict__ Fout, int acc) {
  SITE_PROLOGUE
  if (!s.valid) return;
  const double s0 = __ldg(S + s.n);
  const double s_mt = __ldg(S + at(s, s.x, tm1(s)));
  const double s_mx = __ldg(S + at(s, xm1(s), s.t));
  const double2 F = make_double2(ci.beta * (s0 - s_mt), ci.beta * (s_mx - s0));
  if (Fout) {
    double2 o = F;
    if (acc) {
      const double2 f0 = ld_l2_cg(Fout, s.n);
      o = make_double2(f0.x + F.x, f0.y + F.y);
    }
    st_l2(Fout, s.n, o);
  }
  if (p) {
    const double2 p0 = ld_l2_cg(p, s.n);
    st_l2(p, s.n, make_double2(p0.x - eps * F.x, p0.y - eps * F.y));
  }
}

// p -= eps f and/or Fout (=, or +=) f, f of Eq. force_fermion:
//   f(n, mu) = -Im[ chi^dag(n)(1 - s_mu) U_mu(n) xi(n+mu) - chi^dag(n+mu)(1 + s_mu) U_mu^*(n) xi(n) ].
__global__ void __launch_bounds__(kBlock) k_fermion_kick(Geo g, const double* __restrict__ U,
                                                         const double* __restrict__ chi,
                                                         const double* __restrict__ xi,
                                                         double* __restrict__ p, double eps,
                                                         double* __restrict__ Fout, int acc) {
  SITE_PROLOGUE
  if (!s.valid) return;
  const long long nx = at(s, xp1(s), s.t), nt = at(s, s.x, tp1(s));
  const Lk<double> u = ld_lk(U, s.n);
  const Sp<double> c0 = ld_sp(chi, s.n), x0 = ld_sp(xi, s.n);
  Cx<double> A, B;
  bilinear_x(c0, ld_sp(chi, nx), x0, ld_sp(xi, nx), u.x, A, B);
  const double fx = -(A.im - B.im);
  bilinear_t(c0, ld_sp(chi, nt), x0, ld_sp(xi, nt), u.t, A, B);
  const double ft = -(A.im - B.im);
  if (Fout) {
    double2 o = make_double2(fx, ft);
    if (acc) {
      const double2 f0 = ld_l2_cg(Fout, s.n);
      o = make_double2(f0.x + fx, f0.y + ft);
    }
    st_l2(Fout, s.n, o);
  }
  if (p) {
    const double2 p0 = ld_l2_cg(p, s.n);
    st_l2(p, s.n, make_double2(p0.x - eps * fx, p0.y - eps * ft));
  }
}

// Directional derivative of the hopping term along the link field v:
// out = -1/2 sum_mu (hops of D, or of D^dag) with links W_mu(n) = i v_mu(n) U_mu(n).
// With in = xi (D) this is sum_{m,nu} v(m,nu) w_{2,m,nu}; with in = chi (D^dag)
// it is sum_{m,nu} v(m,nu) w_{1,m,nu} (Sec. 3.1, the vectors w_1, w_2; the
// source sums of Eq. Z12).
template <bool DAG>
__global__ void __launch_bounds__(kBlock) k_deriv_hop(Geo g, const double* __restrict__ U,
                                                      const double* __restrict__ v,
                                                      const double* __restrict__ in,
                                                      double* __restrict__ out) {
  SITE_PROLOGUE
  if (!s.valid) return;
  const int xp = xp1(s), xm = xm1(s), tp = tp1(s), tm = tm1(s);
  const long long nxm = at(s, xm, s.t), ntm = at(s, s.x, tm);
  const Lk<double> u = ld_lk(U, s.n);
  const double2 vn = ld_l2(v, s.n);
  const Cx<double> wx = mul_i(vn.x * u.x), wt = mul_i(vn.y * u.t);
  const Cx<double> wxm = mul_i(ld_l2(v, nxm).x * link_x(U, nxm));
  const Cx<double> wtm = mul_i(ld_l2(v, ntm).y * link_t(U, ntm));
  const Sp<double> o = hop_sum<DAG, double>(ld_sp(in, at(s, xp, s.t)), ld_sp(in, nxm),
                                            ld_sp(in, at(s, s.x, tp)), ld_sp(in, ntm), wx, wxm,
                                            wt, wtm);
  st_sp(out, s.n, -0.5 * o);
}

// Force-gradient assembly for the fermion action (Eq. CFF with f -> v):
//   C(n,mu) = 4 Re[ Z1^dag w_{2,n,mu} + w_{1,n,mu}^dag Z2 - chi^dag d2D xi v(n,mu) ]
// which in terms of the link bilinears A(a,b), B(a,b) of the fermion force is
//   C = 2 Im[A(Z1,xi) - B(Z1,xi) + A(chi,Z2) - B(chi,Z2)] - 2 v Re[A(chi,xi) + B(chi,xi)].
// Z1 is z1 - z1s when z1s is not NULL (z1 = D Z2 from the solver, z1s = s2).
__global__ void __launch_bounds__(kBlock) k_fg_assemble(Geo g, const double* __restrict__ U,
                                                        const double* __restrict__ chi,
                                                        const double* __restrict__ xi,
                                                        const double* __restrict__ z1,
                                                        const double* __restrict__ z1s,
                                                        const double* __restrict__ z2,
                                                        const double* __restrict__ v,
                                                        double* __restrict__ C, int acc) {
  SITE_PROLOGUE
  if (!s.valid) return;
  const long long nb[2] = {at(s, xp1(s), s.t), at(s, s.x, tp1(s))};
  const Lk<double> u = ld_lk(U, s.n);
  const Sp<double> c0 = ld_sp(chi, s.n), x0 = ld_sp(xi, s.n);
  auto ldz1 = [&](long long n) { return z1s ? ld_sp(z1, n) - ld_sp(z1s, n) : ld_sp(z1, n); };
  const Sp<double> a0 = ldz1(s.n), b0 = ld_sp(z2, s.n);
  const double2 vn = ld_l2(v, s.n);
  double out[2];
#pragma unroll
  for (int mu = 0; mu < 2; ++mu) {
    const Sp<double> c1 = ld_sp(chi, nb[mu]), x1 = ld_sp(xi, nb[mu]);
    const Sp<double> a1 = ldz1(nb[mu]), b1 = ld_sp(z2, nb[mu]);
    Cx<double> A0, B0, A1, B1, A2, B2;
    if (mu == 0) {
      bilinear_x(c0, c1, x0, x1, u.x, A0, B0);
      bilinear_x(a0, a1, x0, x1, u.x, A1, B1);
      bilinear_x(c0, c1, b0, b1, u.x, A2, B2);
    } else {
      bilinear_t(c0, c1, x0, x1, u.t, A0, B0);
      bilinear_t(a0, a1, x0, x1, u.t, A1, B1);
      bilinear_t(c0, c1, b0, b1, u.t, A2, B2);
    }
    const double vm = mu == 0 ? vn.x : vn.y;
    out[mu] = 2.0 * ((A1.im - B1.im) + (A2.im - B2.im)) - 2.0 * vm * (A0.re + B0.re);
  }
  double2 o = make_double2(out[0], out[1]);
  if (acc) {
    const double2 c = ld_l2_cg(C, s.n);
    o = make_double2(c.x + o.x, c.y + o.y);
  }
  st_l2(C, s.n, o);
}

// 2 (Hess S_G) v, the C_FG closed form of Sec. 3.1 with f -> v:
//   2 beta [ (v(n,mu) + v(n+mu,nu) - v(n+nu,mu) - v(n,nu)) Re P1
//          + (v(n,mu) - v(n+mu-nu,nu) - v(n-nu,mu) + v(n-nu,nu)) Re P2 ],
// with Re P1 = cos th(n) and Re P2 = cos th(n-nu) for both mu.
// v = F_G gives C_GG.
__global__ void __launch_bounds__(kBlock) k_gauge_hvp(Geo g, const double* __restrict__ q,
                                                      const double* __restrict__ v,
                                                      double* __restrict__ C, int acc) {
  SITE_PROLOGUE
  if (!s.valid) return;
  const GaugeNb b = gauge_nb(s);
  const double2 q0 = ld_l2(q, b.n), qx = ld_l2(q, b.nx), qt = ld_l2(q, b.nt);
  const double2 qmt = ld_l2(q, b.nmt), qxmt = ld_l2(q, b.nxmt);
  const double2 qmx = ld_l2(q, b.nmx), qmxt = ld_l2(q, b.nmxt);
  const double c0 = cos(plaq_angle(q0, qx, qt));
  const double c_mt = cos(plaq_angle(qmt, qxmt, q0));
  const double c_mx = cos(plaq_angle(qmx, q0, qmxt));
  const double2 v0 = ld_l2(v, b.n), vx = ld_l2(v, b.nx), vt = ld_l2(v, b.nt);
  const double2 vmt = ld_l2(v, b.nmt), vxmt = ld_l2(v, b.nxmt);
  const double2 vmx = ld_l2(v, b.nmx), vmxt = ld_l2(v, b.nmxt);
  const double cx = 2.0 * ci.beta *
                    ((v0.x + vx.y - vt.x - v0.y) * c0 + (v0.x - vxmt.y - vmt.x + vmt.y) * c_mt);
  const double ct = 2.0 * ci.beta *
                    ((v0.y + vt.x - vx.y - v0.x) * c0 + (v0.y - vmxt.x - vmx.y + vmx.x) * c_mx);
  double2 o = make_double2(cx, ct);
  if (acc) {
    const double2 cc = ld_l2_cg(C, s.n);
    o = make_double2(cc.x + o.x, cc.y + o.y);
  }
  st_l2(C, s.n, o);
}

// y = w + a x + b z on real link fields (w, z may be NULL: zero).
__global__ void __launch_bounds__(kBlock) k_lincomb(Geo g, double* y, const double* w, double a,
                                                   const double* x, double b, const double* z) {
  SITE_PROLOGUE
  if (!s.valid) return;
  double2 r = w ? ld_l2_cg(w, s.n) : make_double2(0.0, 0.0);
  const double2 xv = ld_l2_cg(x, s.n);
  r.x += a * xv.x;
  r.y += a * xv.y;
  if (z) {
    const double2 zv = ld_l2_cg(z, s.n);
    r.x += b * zv.x;
    r.y += b * zv.y;
  }
  st_l2(y, s.n, r);
}

// Spinors: y = w + a x.
__global__ void __launch_bounds__(kBlock) k_spinor_lincomb(Geo g, double* y, const double* w,
                                                           double a, const double* x) {
  SITE_PROLOGUE
  if (!s.valid) return;
  st_sp(y, s.n, ld_sp_cg(w, s.n) + a * ld_sp_cg(x, s.n));
}

// dst = src on the chains whose mask is nonzero.
__global__ void __launch_bounds__(kBlock) k_copy_masked(Geo g, double* dst, const double* src,
                                                        const int* mask) {
  SITE_PROLOGUE
  if (!s.valid || !mask[c_]) return;
  st_l2(dst, s.n, ld_l2_cg(src, s.n));
}

// Per-chain FP64 sums: K = 1/2 sum p^2, S_G = beta sum (1 - cos th),
// S_F = Re sum phi^dag xi.  Missing inputs contribute zero.
__global__ void __launch_bounds__(kBlock) k_energies(Geo g, const double* __restrict__ q,
                                                     const double* __restrict__ p,
                                                     const double* __restrict__ phi,
                                                     const double* __restrict__ xi,
                                                     double* partials, unsigned* counters,
                                                     double* K, double* SG, double* SF) {
  SITE_PROLOGUE
  double v[3] = {0.0, 0.0, 0.0};
  if (s.valid) {
    if (p) {
      const double2 pv = ld_l2(p, s.n);
      v[0] = 0.5 * (pv.x * pv.x + pv.y * pv.y);
    }
    if (q) {
      const double2 q0 = ld_l2(q, s.n), qx = ld_l2(q, at(s, xp1(s), s.t)),
                    qt = ld_l2(q, at(s, s.x, tp1(s)));
      v[1] = ci.beta * (1.0 - cos(plaq_angle(q0, qx, qt)));
    }
    if (phi && xi) v[2] = redot(ld_sp(phi, s.n), ld_sp(xi, s.n));
  }
  double tot[3];
  if (chain_reduce<3>(v, partials, counters, g, ci, c_, tot) && threadIdx.x == 0) {
    if (K) K[c_] = tot[0];
    if (SG) SG[c_] = tot[1];
    if (SF) SF[c_] = tot[2];
  }
}

// ------------------------------------------------------------ launchers ---

template <typename R>
int launch_dslash(Ctx& c, const R* U, const R* in, R* out, bool dagger, const R* add,
                  double add_scale) {
  if (dagger)
    k_dslash<R, true><<<c.grid(), kBlock, 0, c.s>>>(c.g, U, in, out, add, (R)add_scale);
  else
    k_dslash<R, false><<<c.grid(), kBlock, 0, c.s>>>(c.g, U, in, out, add, (R)add_scale);
  return launched(c.st, "dslash");
}
template int launch_dslash<double>(Ctx&, const double*, const double*, double*, bool,
                                   const double*, double);
template int launch_dslash<float>(Ctx&, const float*, const float*, float*, bool, const float*,
                                  double);

int launch_links(Ctx& c, const double* q, double* U64, float* U32) {
  k_links<<<c.grid(), kBlock, 0, c.s>>>(c.g, q, U64, U32);
  return launched(c.st, "links");
}
int launch_gauge_kick(Ctx& c, const double* q, double* p, double eps, double* Fout, bool acc) {
  if (!c.w.sinp) {  // no workspace (sm_gauge_force): the one-pass form, F only
    if (p || acc || !Fout) return fail(SM_ERR_ARG, "gauge kick without a workspace");
    k_gauge_kick_direct<<<c.grid(), kBlock, 0, c.s>>>(c.g, q, Fout);
    return launched(c.st, "gauge_kick_direct");
  }
  k_plaq_sin<<<c.grid(), kBlock, 0, c.s>>>(c.g, q, c.w.sinp);
  const int rc = launched(c.st, "plaq_sin");
  if (rc) return rc;
  k_gauge_kick<<<c.grid(), kBlock, 0, c.s>>>(c.g, c.w.sinp, p, eps, Fout, acc ? 1 : 0);
  return launched(c.st, "gauge_kick");
}
int launch_fermion_kick(Ctx& c, const double* U64, const double* chi, const double* xi, double* p,
                        double eps, double* Fout, bool acc) {
  k_fermion_kick<<<c.grid(), kBlock, 0, c.s>>>(c.g, U64, chi, xi, p, eps, Fout, acc ? 1 : 0);
  return launched(c.st, "fermion_kick");
}
int launch_deriv_hop(Ctx& c, const double* U64, const double* v, const double* in, double* out,
                     bool dagger) {
  if (dagger)
    k_deriv_hop<true><<<c.grid(), kBlock, 0, c.s>>>(c.g, U64, v, in, out);
  else
    k_deriv_hop<false><<<c.grid(), kBlock, 0, c.s>>>(c.g, U64, v, in, out);
  return launched(c.st, "deriv_hop");
}
int launch_fg_assemble(Ctx& c, const double* U64, const double* chi, const double* xi,
                       const double* z1, const double* z1s, const double* z2, const double* v,
                       double* C, bool acc) {
  k_fg_assemble<<<c.grid(), kBlock, 0, c.s>>>(c.g, U64, chi, xi, z1, z1s, z2, v, C, acc ? 1 : 0);
  return launched(c.st, "fg_assemble");
}
int launch_gauge_hvp(Ctx& c, const double* q, const double* v, double* C, bool acc) {
  k_gauge_hvp<<<c.grid(), kBlock, 0, c.s>>>(c.g, q, v, C, acc ? 1 : 0);
  return launched(c.st, "gauge_hvp");
}
int launch_axpy_links(Ctx& c, double* y, const double* x, double a, const double* z, double b) {
  k_lincomb<<<c.grid(), kBlock, 0, c.s>>>(c.g, y, y, a, x, b, z);
  return launched(c.st, "lincomb");
}
int launch_lincomb(Ctx& c, double* y, const double* w, double a, const double* x, double b,
                   const double* z) {
  k_lincomb<<<c.grid(), kBlock, 0, c.s>>>(c.g, y, w, a, x, b, z);
  return launched(c.st, "lincomb");
}
int launch_spinor_lincomb(Ctx& c, double* y, const double* w, double a, const double* x) {
  k_spinor_lincomb<<<c.grid(), kBlock, 0, c.s>>>(c.g, y, w, a, x);
  return launched(c.st, "spinor_lincomb");
}
int launch_drift(Ctx& c, double* q, const double* p, double eps) {
  k_lincomb<<<c.grid(), kBlock, 0, c.s>>>(c.g, q, q, eps, p, 0.0, nullptr);
  return launched(c.st, "drift");
}
int launch_energies(Ctx& c, const double* q, const double* p, const double* phi, const double* xi,
                    double* K, double* SG, double* SF) {
  k_energies<<<c.grid(), kBlock, 0, c.s>>>(c.g, q, p, phi, xi, c.w.partials, c.w.counters, K, SG,
                                          SF);
  return launched(c.st, "energies");
}
int launch_copy_links_masked(Ctx& c, double* dst, const double* src, const int* mask) {
  k_copy_masked<<<c.grid(), kBlock, 0, c.s>>>(c.g, dst, src, mask);
  return launched(c.st, "copy_masked");
}

}  // namespace sm

// ============================================================== C ABI =====

using namespace sm;

extern "C" {

const char* sm_last_error(void) { return sm::g_err; }
int sm_version(void) { return 1; }
long long sm_launch_count(void) { return sm::g_launches.load(); }

int sm_lattice_create(int nchains, const int* L, const int* T, const double* beta,
                      const double* m0, sm_lattice** out) {
  if (!out) return fail(SM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nchains < 1) return fail(SM_ERR_ARG, "nchains = %d < 1", nchains);
  if (!L || !T || !beta || !m0) return fail(SM_ERR_ARG, "NULL size or coupling array");
  sm_lattice* lat = new sm_lattice();
  lat->nchains = nchains;
  lat->chains.resize(nchains);
  long long off = 0;
  int blk = 0;
  std::vector<int> blk_chain;
  for (int c = 0; c < nchains; ++c) {
    if (L[c] < 2 || T[c] < 2 || (long long)L[c] * T[c] > (1LL << 30)) {
      delete lat;
      return fail(SM_ERR_ARG, "chain %d: bad lattice %d x %d (sides >= 2, volume <= 2^30)", c,
                  L[c], T[c]);
    }
    ChainInfo& ci = lat->chains[c];
    ci.L = L[c];
    ci.T = T[c];
    ci.off = off;
    ci.beta = beta[c];
    ci.m0 = m0[c];
    const long long V = (long long)L[c] * T[c];
    ci.nblk = (int)((V + kBlock - 1) / kBlock);
    ci.blk0 = blk;
    for (int b = 0; b < ci.nblk; ++b) blk_chain.push_back(c);
    blk += ci.nblk;
    off += V;
  }
  if (blk > (1 << 30)) {
    delete lat;
    return fail(SM_ERR_ARG, "batch too large");
  }
  lat->N = off;
  lat->nblocks = blk;
  big_tile_ranges(lat);
  lat->cg_variant = -1;
  lat->tma_spin = kTmaSpin;
  cudaGetDevice(&lat->device);
  if (const int rc = stream_ranges(lat)) {
    delete lat;
    return rc;
  }
  cudaError_t e = cudaMalloc(&lat->d_chains, sizeof(ChainInfo) * nchains);
  if (e == cudaSuccess) e = cudaMalloc(&lat->d_blk_chain, sizeof(int) * blk);
  if (e == cudaSuccess) e = cudaMalloc(&lat->d_chain_list, sizeof(int) * nchains);
  if (e == cudaSuccess) {
    std::vector<int> ids(nchains);
    for (int i = 0; i < nchains; ++i) ids[i] = i;
    e = cudaMemcpy(lat->d_chain_list, ids.data(), sizeof(int) * nchains, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(lat->d_chains, lat->chains.data(), sizeof(ChainInfo) * nchains,
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(lat->d_blk_chain, blk_chain.data(), sizeof(int) * blk, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaHostAlloc(&lat->h_pinned, 64 * sizeof(int), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lat->ev[0], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lat->ev[1], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    sm_lattice_destroy(lat);
    return fail(SM_ERR_CUDA, "lattice tables: %s", cudaGetErrorString(e));
  }
  const int rc = build_tile_table(lat);
  if (rc) {
    sm_lattice_destroy(lat);
    return rc;
  }
  // mixed batches: which chains fit the chain-resident kernel, which the
  // 4-block cluster kernel, and which take the grid-wide path
  std::vector<int> small, big;
  lat->grid_mask.assign(nchains, 1);
  for (int c = 0; c < nchains; ++c) {
    if (lat->chains[c].L * lat->chains[c].T <= 4096) {
      small.push_back(c);
      lat->grid_mask[c] = 0;
    } else if (big_chain_shape(lat->chains[c])) {
      big.push_back(c);
    }
  }
  lat->nsmall = (small.size() < (size_t)nchains) ? (int)small.size() : 0;
  lat->nbig = (small.size() + big.size() == (size_t)nchains) ? (int)big.size() : 0;
  e = cudaMalloc(&lat->d_big_list, sizeof(int) * (big.empty() ? 1 : big.size()));
  if (e == cudaSuccess && !big.empty())
    e = cudaMemcpy(lat->d_big_list, big.data(), sizeof(int) * big.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&lat->d_grid_mask, nchains);
  if (e == cudaSuccess) e = cudaMalloc(&lat->d_small_list, sizeof(int) * (small.empty() ? 1 : small.size()));
  if (e == cudaSuccess)
    e = cudaMemcpy(lat->d_grid_mask, lat->grid_mask.data(), nchains, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !small.empty())
    e = cudaMemcpy(lat->d_small_list, small.data(), sizeof(int) * small.size(), cudaMemcpyHostToDevice);
  // the chains of at most 4096 sites by kernel group, each group's chains
  // in batch order
  {
    std::vector<int> glist;
    lat->ngroups = 0;
    for (int kind = 0; kind < sm_lattice::kGroups; ++kind) {
      const int begin = (int)glist.size();
      int vmax = 0;
      for (int c : small)
        if (chain_group_kind(lat->chains[c]) == kind) {
          glist.push_back(c);
          vmax = std::max(vmax, lat->chains[c].L * lat->chains[c].T);
        }
      if ((int)glist.size() > begin) {
        const int g = lat->ngroups++;
        lat->group_kind[g] = kind;
        lat->group_begin[g] = begin;
        lat->group_count[g] = (int)glist.size() - begin;
        lat->group_vmax[g] = vmax;
      }
    }
    if (e == cudaSuccess) e = cudaMalloc(&lat->d_group_list, sizeof(int) * (glist.empty() ? 1 : glist.size()));
    if (e == cudaSuccess && !glist.empty())
      e = cudaMemcpy(lat->d_group_list, glist.data(), sizeof(int) * glist.size(),
                     cudaMemcpyHostToDevice);
    for (int g = 1; g < lat->ngroups && e == cudaSuccess; ++g) {
      e = cudaStreamCreateWithFlags(&lat->gstream[g], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lat->gev_join[g], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lat->gev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&lat->nsm, cudaDevAttrMultiProcessorCount, lat->device);
  }
  if (e == cudaSuccess) e = cudaMalloc(&lat->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(lat->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&lat->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lat->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lat->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    sm_lattice_destroy(lat);
    return fail(SM_ERR_CUDA, "lattice tables: %s", cudaGetErrorString(e));
  }
  *out = lat;
  return SM_OK;
}

int sm_lattice_destroy(sm_lattice* lat) {
  if (!lat) return SM_OK;
  if (lat->d_chains) cudaFree(lat->d_chains);
  if (lat->d_blk_chain) cudaFree(lat->d_blk_chain);
  if (lat->d_chain_list) cudaFree(lat->d_chain_list);
  if (lat->d_tiles) cudaFree(lat->d_tiles);
  if (lat->d_grid_mask) cudaFree(lat->d_grid_mask);
  if (lat->d_err) cudaFree(lat->d_err);
  if (lat->d_small_list) cudaFree(lat->d_small_list);
  if (lat->d_big_list) cudaFree(lat->d_big_list);
  if (lat->side) cudaStreamDestroy(lat->side);
  if (lat->heavy) sm_lattice_destroy(lat->heavy);
  if (lat->d_group_list) cudaFree(lat->d_group_list);
  for (int g = 0; g < sm_lattice::kGroups; ++g) {
    if (lat->gstream[g]) cudaStreamDestroy(lat->gstream[g]);
    if (lat->gev_join[g]) cudaEventDestroy(lat->gev_join[g]);
  }
  if (lat->gev_fork) cudaEventDestroy(lat->gev_fork);
  if (lat->ev_fork) cudaEventDestroy(lat->ev_fork);
  if (lat->ev_join) cudaEventDestroy(lat->ev_join);
  if (lat->d_tiles_big) cudaFree(lat->d_tiles_big);
  if (lat->d_stream) cudaFree(lat->d_stream);
  if (lat->d_stream_cg) cudaFree(lat->d_stream_cg);
  if (lat->h_pinned) cudaFreeHost(lat->h_pinned);
  if (lat->ev[0]) cudaEventDestroy(lat->ev[0]);
  if (lat->ev[1]) cudaEventDestroy(lat->ev[1]);
  delete lat;
  return SM_OK;
}

long long sm_lattice_sites(const sm_lattice* lat) { return lat ? lat->N : 0; }

int sm_lattice_check(const sm_lattice* lat, int* code) {
  if (!lat || !code) return fail(SM_ERR_ARG, "sm_lattice_check: NULL argument");
  int h = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, lat->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(lat->d_err, 0, sizeof(int));
  if (e == cudaSuccess && lat->heavy) {  // the heavy copy's kernels record there
    int hh = 0;
    e = cudaMemcpy(&hh, lat->heavy->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(lat->heavy->d_err, 0, sizeof(int));
    h |= hh;
  }
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "sm_lattice_check: %s", cudaGetErrorString(e));
  *code = h;
  if (h) return fail(SM_ERR_TIMEOUT, "a bounded device-side wait gave up (code %d)", h);
  return SM_OK;
}
int sm_debug_read(long long* violations, long long* first_index, int* first_where) {
  if (!violations || !first_index || !first_where)
    return fail(SM_ERR_ARG, "sm_debug_read: NULL argument");
  *violations = 0;
  *first_index = -1;
  *first_where = -1;
#ifdef SM_DEBUG
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "sm_debug_read: %s", cudaGetErrorString(e));
  unsigned long long n = 0;
  for (const dbg::Hooks& h : dbg::hooks()) h.take(&n, first_index, first_where);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "sm_debug_read: %s", cudaGetErrorString(e));
  *violations = (long long)n;
  return SM_OK;
#else
  *first_where = -2;  // the checks are not compiled into this library
  return SM_OK;
#endif
}

int sm_lattice_set_heavy(sm_lattice* lat, double dm) {
  if (!lat) return fail(SM_ERR_ARG, "sm_lattice_set_heavy: lattice is NULL");
  if (!(dm > 0.0) || !std::isfinite(dm))
    return fail(SM_ERR_ARG, "sm_lattice_set_heavy: dm must be positive and finite");
  const int n = lat->nchains;
  std::vector<int> L(n), T(n);
  std::vector<double> beta(n), m0(n);
  for (int c = 0; c < n; ++c) {
    L[c] = lat->chains[c].L;
    T[c] = lat->chains[c].T;
    beta[c] = lat->chains[c].beta;
    m0[c] = lat->chains[c].m0 + dm;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && dev != lat->device) e = cudaSetDevice(lat->device);
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "sm_lattice_set_heavy: %s", cudaGetErrorString(e));
  sm_lattice* h = nullptr;
  const int rc = sm_lattice_create(n, L.data(), T.data(), beta.data(), m0.data(), &h);
  if (dev != lat->device) cudaSetDevice(dev);
  if (rc) return rc;
  h->cg_variant = lat->cg_variant;
  if (lat->heavy) sm_lattice_destroy(lat->heavy);
  lat->heavy = h;
  lat->heavy_dm = dm;
  return SM_OK;
}

int sm_set_wait_limit(sm_lattice* lat, int polls) {
  if (!lat) return fail(SM_ERR_ARG, "sm_set_wait_limit: lattice is NULL");
  if (polls < -1 || polls > kTmaSpin)
    return fail(SM_ERR_ARG, "sm_set_wait_limit: polls must be -1 or in [0, %d]", kTmaSpin);
  lat->tma_spin = polls < 0 ? kTmaSpin : polls;
  return SM_OK;
}
int sm_lattice_chains(const sm_lattice* lat) { return lat ? lat->nchains : 0; }
size_t sm_workspace_bytes(const sm_lattice* lat) { return lat ? Ws::bytes(lat) : 0; }

static bool al16(const void* p) { return ((uintptr_t)p & 15) == 0; }

int sm_links(const sm_lattice* lat, const double* q, double* U64, float* U32, void* stream) {
  Ctx c;
  int rc = c.init(lat, nullptr, 0, stream, nullptr, false);
  if (rc) return rc;
  if (!q || (!U64 && !U32)) return fail(SM_ERR_ARG, "sm_links: NULL field");
  if (!al16(q) || !al16(U64) || !al16(U32)) return fail(SM_ERR_ARG, "sm_links: unaligned field");
  return launch_links(c, q, U64, U32);
}

int sm_apply_D(const sm_lattice* lat, const void* U, const void* in, void* out, int dagger,
               int prec, void* stream) {
  Ctx c;
  int rc = c.init(lat, nullptr, 0, stream, nullptr, false);
  if (rc) return rc;
  if (!U || !in || !out) return fail(SM_ERR_ARG, "sm_apply_D: NULL field");
  if (!al16(U) || !al16(in) || !al16(out)) return fail(SM_ERR_ARG, "sm_apply_D: unaligned field");
  if (in == out) return fail(SM_ERR_ARG, "sm_apply_D: in and out alias");
  if (prec == SM_F64)
    return launch_dslash<double>(c, (const double*)U, (const double*)in, (double*)out, dagger != 0,
                                 nullptr, 0.0);
  if (prec == SM_F32)
    return launch_dslash<float>(c, (const float*)U, (const float*)in, (float*)out, dagger != 0,
                                nullptr, 0.0);
  return fail(SM_ERR_ARG, "sm_apply_D: prec must be SM_F64 or SM_F32");
}

int sm_apply_DdagD(const sm_lattice* lat, const void* U, const void* in, void* out, int prec,
                   void* ws, size_t ws_bytes, void* stream) {
  (void)ws;
  (void)ws_bytes;
  Ctx c;
  int rc = c.init(lat, nullptr, 0, stream, nullptr, false);
  if (rc) return rc;
  if (!U || !in || !out) return fail(SM_ERR_ARG, "sm_apply_DdagD: NULL field");
  if (!al16(U) || !al16(in) || !al16(out))
    return fail(SM_ERR_ARG, "sm_apply_DdagD: unaligned field");
  if (in == out) return fail(SM_ERR_ARG, "sm_apply_DdagD: in and out alias");
  if (prec == SM_F64) return launch_ddagd<double>(c, (const double*)U, (const double*)in, (double*)out);
  if (prec == SM_F32) return launch_ddagd<float>(c, (const float*)U, (const float*)in, (float*)out);
  return fail(SM_ERR_ARG, "sm_apply_DdagD: prec must be SM_F64 or SM_F32");
}

}  // extern "C"
