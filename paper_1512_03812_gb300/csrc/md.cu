// md.cu -- forces, force-gradient terms, energies, the integration schemes of
// Sec. 2 and the HMC trajectory, as host-side sequences of the site kernels
// (core.cu) and CG solves (solver.cu).
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
#define SM_TRY(expr)            \
  do {                          \
    const int rc_ = (expr);     \
    if (rc_ != SM_OK) return rc_; \
  } while (0)

static bool al16(const void* p) { return ((uintptr_t)p & 15) == 0; }

static int check_cg(const sm_cg_params* cg) {
  if (!cg) return fail(SM_ERR_ARG, "cg params are NULL");
  if (cg->prec != SM_F64 && cg->prec != SM_MIXED)
    return fail(SM_ERR_ARG, "cg prec must be SM_F64 or SM_MIXED");
  return SM_OK;
}

static int check_part(int part) {
  if (part < SM_PART_GAUGE || part > SM_PART_FULL) return fail(SM_ERR_ARG, "bad part %d", part);
  return SM_OK;
}

// One part of the determinant split (a call of the single-part entry points).
static int check_split_part(const sm_lattice* L, int part) {
  if (part != SM_PART_HEAVY && part != SM_PART_RATIO) return check_part(part);
  if (!L->heavy) return fail(SM_ERR_ARG, "part %d needs sm_lattice_set_heavy first", part);
  return SM_OK;
}

static bool three_level(int scheme) {
  return scheme == SM_NESTED3_LEAPFROG || scheme == SM_ADAPTED_NESTED3_FG;
}

// The context of the lattice's heavy copy (the same chains at m0 + dm): the
// same stream, statistics and workspace (the heavy copy's carve of the
// buffer gives every common field the same address), its own chain table.
static Ctx heavy_ctx(const Ctx& c) {
  Ctx h = c;
  h.L = c.L->heavy;
  h.g.chains = h.L->d_chains;
  h.g.blk_chain = h.L->d_blk_chain;
  h.chain_flags.clear();
  return h;
}

// Failures of the heavy copy's solves count as the chain's own.
static void merge_flags(Ctx& c, const Ctx& h) {
  if (h.chain_flags.empty()) return;
  if (c.chain_flags.empty()) c.chain_flags.assign(h.chain_flags.size(), 0);
  for (size_t i = 0; i < h.chain_flags.size(); ++i) c.chain_flags[i] |= h.chain_flags[i];
}

// U64 (and U32 for mixed solves) from q.
static int make_links(Ctx& c, const double* q, double* U64, float* U32, const sm_cg_params& cg) {
  return launch_links(c, q, U64, cg.prec == SM_MIXED ? U32 : nullptr);
}

// xi = (D^dag D)^{-1} phi and chi = D xi (Eq. chi_xi_vectors), in c.w.xi, c.w.chi.
// chi comes from the solver where its last FP64 reliable update computed it.
static int chi_xi(Ctx& c, const double* U64, const float* U32, const double* phi,
                  const sm_cg_params& cg) {
  bool have = false;
  SM_TRY(cg_solve(c, U64, U32, phi, c.w.xi, cg, nullptr, nullptr, c.w.chi, &have));
  c.st->inversions += 2;
  c.st->force_evals++;
  return have ? SM_OK : launch_dslash<double>(c, U64, c.w.xi, c.w.chi, false, nullptr, 0.0);
}

// The heavy part: xi = (D_h^dag D_h)^{-1} phi_h and chi = D_h xi in c.w.xi,
// c.w.chi (Eq. chi_xi_vectors at the heavy mass).
static int chi_xi_heavy(Ctx& c, const double* U64, const float* U32, const double* phi_h,
                        const sm_cg_params& cg) {
  Ctx h = heavy_ctx(c);
  bool have = false;
  int rc = cg_solve(h, U64, U32, phi_h, c.w.xi, cg, nullptr, nullptr, c.w.chi, &have);
  merge_flags(c, h);
  if (rc) return rc;
  c.st->inversions += 2;
  c.st->force_evals++;
  return have ? SM_OK : launch_dslash<double>(h, U64, c.w.xi, c.w.chi, false, nullptr, 0.0);
}

// The ratio part: psi = D_h^dag phi_r (c.w.psi), X = (D^dag D)^{-1} psi
// (c.w.xi) and a = D X - phi_r (c.w.chi).  dS_r/dq is the bilinear of
// Eq. force_fermion with chi -> a, xi -> X (the hopping terms of D and D_h
// are the same), and the force-gradient term of S_r is Eq. CFF / Z12 with the
// same substitution.
static int ratio_vectors(Ctx& c, const double* U64, const float* U32, const double* phi_r,
                         const sm_cg_params& cg) {
  Ctx h = heavy_ctx(c);
  SM_TRY(launch_dslash<double>(h, U64, phi_r, c.w.psi, true, nullptr, 0.0));
  bool have = false;
  SM_TRY(cg_solve(c, U64, U32, c.w.psi, c.w.xi, cg, nullptr, nullptr, c.w.chi, &have));
  c.st->inversions += 2;
  c.st->force_evals++;
  if (have) return launch_spinor_lincomb(c, c.w.chi, c.w.chi, -1.0, phi_r);
  return launch_dslash<double>(c, U64, c.w.xi, c.w.chi, false, phi_r, -1.0);
}

// The force of `part` at q (links U64/U32 of q): written to F (if not NULL)
// and/or applied as the kick p -= eps F (if p is not NULL).  phi is the
// pseudofermion of the fermion part (or the ratio part), phi_h the heavy one.
static int force_at(Ctx& c, const double* q, const double* U64, const float* U32,
                    const double* phi, int part, const sm_cg_params& cg, double* F, double* p,
                    double eps, const double* phi_h = nullptr) {
  bool acc = false;  // F holds a part already
  if (part & SM_PART_GAUGE) {
    SM_TRY(launch_gauge_kick(c, q, p, eps, F, false));
    acc = true;
  }
  if (part & SM_PART_FERMION) {
    SM_TRY(chi_xi(c, U64, U32, phi, cg));
    SM_TRY(launch_fermion_kick(c, U64, c.w.chi, c.w.xi, p, eps, F, acc));
    acc = true;
  }
  if (part & SM_PART_HEAVY) {
    SM_TRY(chi_xi_heavy(c, U64, U32, phi_h, cg));
    SM_TRY(launch_fermion_kick(c, U64, c.w.chi, c.w.xi, p, eps, F, acc));
    acc = true;
  }
  if (part & SM_PART_RATIO) {
    SM_TRY(ratio_vectors(c, U64, U32, phi, cg));
    SM_TRY(launch_fermion_kick(c, U64, c.w.chi, c.w.xi, p, eps, F, acc));
  }
  return SM_OK;
}

// C = 2 (Hess S_part) v at q.  For the fermion part chi and xi of q must be in
// c.w.chi and c.w.xi.  The sums over (m, nu) of Eq. Z12 are formed before the
// single inversion:  D^dag D Z2 = D^dag s2 + s1,  Z1 = D Z2 - s2.
static int hess_times(Ctx& c, const double* q, const double* U64, const float* U32, int part,
                      const double* v, const sm_cg_params& cg, double* C) {
  bool acc = false;
  if (part & SM_PART_GAUGE) {
    SM_TRY(launch_gauge_hvp(c, q, v, C, false));
    acc = true;
  }
  if (part & SM_PART_FERMION) {
    SM_TRY(launch_deriv_hop(c, U64, v, c.w.chi, c.w.s1, true));   // sum w_1 v
    SM_TRY(launch_deriv_hop(c, U64, v, c.w.xi, c.w.s2, false));   // sum w_2 v
    SM_TRY(launch_dslash<double>(c, U64, c.w.s2, c.w.b, true, c.w.s1, 1.0));
    // Z1 = D Z2 - s2: D Z2 from the solver where it computed it
    bool have = false;
    SM_TRY(cg_solve(c, U64, U32, c.w.b, c.w.z2, cg, nullptr, nullptr, c.w.z1, &have));
    c.st->inversions += 2;
    if (!have) SM_TRY(launch_dslash<double>(c, U64, c.w.z2, c.w.z1, false, c.w.s2, -1.0));
    SM_TRY(launch_fg_assemble(c, U64, c.w.chi, c.w.xi, c.w.z1, have ? c.w.s2 : nullptr, c.w.z2,
                              v, C, acc));
  }
  return SM_OK;
}

// F of `part` into c.w.F and C = 2 Hess F into C (Eq. force_gradient).
// The ratio part alone (part == SM_PART_RATIO) leaves (a, X) in c.w.chi,
// c.w.xi, where the fermion branch of hess_times reads them.
static int force_and_gradient(Ctx& c, const double* q, const double* U64, const float* U32,
                              const double* phi, int part, const sm_cg_params& cg, double* C) {
  SM_TRY(force_at(c, q, U64, U32, phi, part, cg, c.w.F, nullptr, 0.0));
  return hess_times(c, q, U64, U32, part == SM_PART_RATIO ? SM_PART_FERMION : part, c.w.F, cg,
                    C);
}

// F(q - (h^2/24) F(q)) of `part` into F and/or as the kick p -= eps F.
static int shifted_force(Ctx& c, const double* q, const double* U64, const float* U32,
                         const double* phi, int part, double h, const sm_cg_params& cg, double* F,
                         double* p, double eps, const double* phi_h = nullptr) {
  SM_TRY(force_at(c, q, U64, U32, phi, part, cg, c.w.F, nullptr, 0.0, phi_h));
  SM_TRY(launch_lincomb(c, c.w.qs, q, -h * h / 24.0, c.w.F, 0.0, nullptr));
  if (part & ~SM_PART_GAUGE) SM_TRY(make_links(c, c.w.qs, c.w.U64s, c.w.U32s, cg));
  return force_at(c, c.w.qs, c.w.U64s, c.w.U32s, phi, part, cg, F, p, eps, phi_h);
}

// ------------------------------------------------------------- schedules --

enum OpKind { OP_DRIFT, OP_KICK, OP_FG };
struct Op {
  OpKind k;
  int part;
  double eps;  // drift/kick step; for OP_FG the step h of the force-gradient stage
};

static void inner_lf(std::vector<Op>& o, double h, int M) {
  for (int i = 0; i < M; ++i) {
    o.push_back({OP_KICK, SM_PART_GAUGE, h / (2.0 * M)});
    o.push_back({OP_DRIFT, 0, h / M});
    o.push_back({OP_KICK, SM_PART_GAUGE, h / (2.0 * M)});
  }
}

static void inner_fg(std::vector<Op>& o, double h, int M) {
  const double hm = h / M;
  for (int i = 0; i < M; ++i) {
    o.push_back({OP_KICK, SM_PART_GAUGE, hm / 6.0});
    o.push_back({OP_DRIFT, 0, hm / 2.0});
    o.push_back({OP_FG, SM_PART_GAUGE, hm});
    o.push_back({OP_DRIFT, 0, hm / 2.0});
    o.push_back({OP_KICK, SM_PART_GAUGE, hm / 6.0});
  }
}

// Delta_2(h): M2 leapfrog steps of the heavy part, each with M gauge
// leapfrog steps inside (the middle level of the three-level schemes).
static void middle_lf(std::vector<Op>& o, double h, int M2, int M) {
  for (int i = 0; i < M2; ++i) {
    o.push_back({OP_KICK, SM_PART_HEAVY, h / (2.0 * M2)});
    inner_lf(o, h / M2, M);
    o.push_back({OP_KICK, SM_PART_HEAVY, h / (2.0 * M2)});
  }
}

// The operations of one step of size h, written as the compositions of
// Sec. 2 (Eq. leap, 5stage, 5stage_fg, 11_stage, leap_multi, 5stage_multi,
// 5stage_multi_fg, ad_5stage_multi_fg).
static int build_step(std::vector<Op>& o, const sm_md_params& md, double h) {
  const int F = SM_PART_FULL, Fe = SM_PART_FERMION;
  const double lam = md.lambda;
  const int M = md.M;
  switch (md.scheme) {
    case SM_LEAPFROG:
      o.push_back({OP_KICK, F, h / 2});
      o.push_back({OP_DRIFT, 0, h});
      o.push_back({OP_KICK, F, h / 2});
      return SM_OK;
    case SM_FIVE_STAGE:
      o.push_back({OP_KICK, F, lam * h});
      o.push_back({OP_DRIFT, 0, h / 2});
      o.push_back({OP_KICK, F, (1 - 2 * lam) * h});
      o.push_back({OP_DRIFT, 0, h / 2});
      o.push_back({OP_KICK, F, lam * h});
      return SM_OK;
    case SM_FIVE_STAGE_FG:
      o.push_back({OP_KICK, F, h / 6});
      o.push_back({OP_DRIFT, 0, h / 2});
      o.push_back({OP_FG, F, h});
      o.push_back({OP_DRIFT, 0, h / 2});
      o.push_back({OP_KICK, F, h / 6});
      return SM_OK;
    case SM_NESTED_LEAPFROG:
      o.push_back({OP_KICK, Fe, h / 2});
      inner_lf(o, h, M);
      o.push_back({OP_KICK, Fe, h / 2});
      return SM_OK;
    case SM_NESTED_FIVE_STAGE:
      o.push_back({OP_KICK, Fe, lam * h});
      inner_lf(o, h / 2, M);
      o.push_back({OP_KICK, Fe, (1 - 2 * lam) * h});
      inner_lf(o, h / 2, M);
      o.push_back({OP_KICK, Fe, lam * h});
      return SM_OK;
    case SM_NESTED_FG:
      o.push_back({OP_KICK, Fe, h / 6});
      inner_fg(o, h / 2, M);
      o.push_back({OP_FG, Fe, h});
      inner_fg(o, h / 2, M);
      o.push_back({OP_KICK, Fe, h / 6});
      return SM_OK;
    case SM_ADAPTED_NESTED_FG:
      o.push_back({OP_KICK, Fe, h / 6});
      inner_lf(o, h / 2, M);
      o.push_back({OP_FG, Fe, h});
      inner_lf(o, h / 2, M);
      o.push_back({OP_KICK, Fe, h / 6});
      return SM_OK;
    case SM_ELEVEN_STAGE: {
      // force weights s, l, (1 - 2 (l + s)) / 2 (twice), l, s; drift weights
      // e, t, 1 - 2 (t + e), t, e (Eq. 11_stage; the weights are those of
      // Eq. (71) of Omelyan, Mryglod and Folk, 2003, cited by the paper)
      const double s = 0.08398315262876693, e = 0.2539785108410595;
      const double l = 0.6822365335719091, t = -0.03230286765269967;
      const double mb = 0.5 * (1.0 - 2.0 * (l + s)), ma = 1.0 - 2.0 * (t + e);
      const double kw[6] = {s, l, mb, mb, l, s}, dw[5] = {e, t, ma, t, e};
      for (int k = 0; k < 6; ++k) {
        o.push_back({OP_KICK, F, kw[k] * h});
        if (k < 5) o.push_back({OP_DRIFT, 0, dw[k] * h});
      }
      return SM_OK;
    }
    case SM_NESTED3_LEAPFROG: {
      const int R = SM_PART_RATIO;
      o.push_back({OP_KICK, R, h / 2});
      middle_lf(o, h, md.M2, M);
      o.push_back({OP_KICK, R, h / 2});
      return SM_OK;
    }
    case SM_ADAPTED_NESTED3_FG: {
      const int R = SM_PART_RATIO;
      o.push_back({OP_KICK, R, h / 6});
      middle_lf(o, h / 2, md.M2, M);
      o.push_back({OP_FG, R, h});
      middle_lf(o, h / 2, md.M2, M);
      o.push_back({OP_KICK, R, h / 6});
      return SM_OK;
    }
    default:
      return fail(SM_ERR_ARG, "unknown scheme %d", md.scheme);
  }
}

// Adjacent kicks of the same part at the same links are one kick.
static void merge(std::vector<Op>& o) {
  std::vector<Op> m;
  for (const Op& op : o) {
    if (!m.empty() && op.k == OP_KICK && m.back().k == OP_KICK && m.back().part == op.part)
      m.back().eps += op.eps;
    else
      m.push_back(op);
  }
  o.swap(m);
}

static int check_md(const sm_md_params* md, const sm_lattice* L = nullptr) {
  if (!md) return fail(SM_ERR_ARG, "md params are NULL");
  if (md->scheme < SM_LEAPFROG || md->scheme > SM_ADAPTED_NESTED3_FG)
    return fail(SM_ERR_ARG, "unknown scheme %d", md->scheme);
  if (three_level(md->scheme)) {
    if (md->M2 < 1) return fail(SM_ERR_ARG, "M2 = %d < 1", md->M2);
    if (L && !L->heavy)
      return fail(SM_ERR_ARG, "three-level schemes need sm_lattice_set_heavy first");
  }
  if (md->M < 1) return fail(SM_ERR_ARG, "M = %d < 1", md->M);
  if (md->fg != SM_FG_EXACT && md->fg != SM_FG_SHIFTED) return fail(SM_ERR_ARG, "bad fg mode");
  if (md->sf_start != SM_SF_SOLVE && md->sf_start != SM_SF_NOISE)
    return fail(SM_ERR_ARG, "bad sf_start %d", md->sf_start);
  return check_cg(&md->cg);
}

// The NVTX name of an operation (one range per operation of a schedule).
static const char* op_name(const Op& op) {
  if (op.k == OP_DRIFT) return "md:drift";
  const bool fg = op.k == OP_FG;
  switch (op.part) {
    case SM_PART_GAUGE: return fg ? "md:fg gauge" : "md:kick gauge";
    case SM_PART_FERMION: return fg ? "md:fg fermion" : "md:kick fermion";
    case SM_PART_HEAVY: return fg ? "md:fg heavy" : "md:kick heavy";
    case SM_PART_RATIO: return fg ? "md:fg ratio" : "md:kick ratio";
    default: return fg ? "md:fg full" : "md:kick full";
  }
}

// Executes `ops` on (q, p).  Links are refreshed lazily, only before an
// operation that needs the fermion force.
static int execute(Ctx& c, const std::vector<Op>& ops, double* q, double* p, const double* phi,
                   const sm_md_params& md, const double* phi_h) {
  bool links_ok = false;
  const sm_cg_params& cg = md.cg;
  for (const Op& op : ops) {
    Range range(op_name(op));
    if ((op.k != OP_DRIFT) && (op.part & ~SM_PART_GAUGE) && !links_ok) {
      SM_TRY(make_links(c, q, c.w.U64, c.w.U32, cg));
      links_ok = true;
    }
    switch (op.k) {
      case OP_DRIFT:
        SM_TRY(launch_drift(c, q, p, op.eps));
        links_ok = false;
        break;
      case OP_KICK:
        SM_TRY(force_at(c, q, c.w.U64, c.w.U32, phi, op.part, cg, nullptr, p, op.eps, phi_h));
        break;
      case OP_FG: {
        // e^{(2/3) h B + (1/72) h^3 C}:  p <- p - (2h/3) F + (h^3/72) C
        const double h = op.eps;
        if (md.fg == SM_FG_EXACT) {
          SM_TRY(force_and_gradient(c, q, c.w.U64, c.w.U32, phi, op.part, cg, c.w.C));
          SM_TRY(launch_lincomb(c, p, p, -2.0 * h / 3.0, c.w.F, h * h * h / 72.0, c.w.C));
        } else {
          SM_TRY(shifted_force(c, q, c.w.U64, c.w.U32, phi, op.part, h, cg, nullptr, p,
                               2.0 * h / 3.0, phi_h));
        }
        break;
      }
    }
  }
  return SM_OK;
}

// phi: the pseudofermion; for the three-level schemes phi_r, with phi_h
// given separately (phi_h NULL: phi holds [phi_r; phi_h]).
static int md_run(Ctx& c, double* q, double* p, const double* phi, const sm_md_params& md,
                  double h, int nsteps, const double* phi_h = nullptr) {
  std::vector<Op> ops;
  for (int i = 0; i < nsteps; ++i) SM_TRY(build_step(ops, md, h));
  if (md.merge_kicks) merge(ops);
  if (three_level(md.scheme) && !phi_h) phi_h = phi + 4 * (size_t)c.L->N;
  return execute(c, ops, q, p, phi, md, phi_h);
}

}  // namespace sm

// ============================================================== C ABI =====

using namespace sm;

// The error code for chains whose solves failed during a trajectory.
static int chain_failures(const Ctx& c, const char* who) {
  int nan = 0, nc = 0;
  for (int f : c.chain_flags) {
    nan += (f & 2) != 0;
    nc += (f & 1) != 0;
  }
  if (nan) return fail(SM_ERR_NAN, "%s: %d chain(s) hit a non-finite value", who, nan);
  if (nc) return fail(SM_ERR_NOT_CONVERGED, "%s: CG reached maxit on %d chain(s)", who, nc);
  return SM_OK;
}

static int fields_ok(std::initializer_list<const void*> ps, const char* who) {
  for (const void* p : ps) {
    if (!p) return fail(SM_ERR_ARG, "%s: NULL field", who);
    if (!al16(p)) return fail(SM_ERR_ARG, "%s: field not 16-byte aligned", who);
  }
  return SM_OK;
}

extern "C" {

int sm_gauge_force(const sm_lattice* lat, const double* q, double* F, void* stream) {
  Ctx c;
  SM_TRY(c.init(lat, nullptr, 0, stream, nullptr, false));
  SM_TRY(fields_ok({q, F}, "sm_gauge_force"));
  return launch_gauge_kick(c, q, nullptr, 0.0, F, false);
}

int sm_force(const sm_lattice* lat, const double* q, const double* phi, int part,
             const sm_cg_params* cg, double* F, void* ws, size_t ws_bytes, sm_stats* stats,
             void* stream) {
  Ctx c;
  SM_TRY(c.init(lat, ws, ws_bytes, stream, stats));
  SM_TRY(check_split_part(lat, part));
  SM_TRY(fields_ok({q, F}, "sm_force"));
  if (part & ~SM_PART_GAUGE) {
    SM_TRY(check_cg(cg));
    SM_TRY(fields_ok({phi}, "sm_force"));
    SM_TRY(make_links(c, q, c.w.U64, c.w.U32, *cg));
  }
  sm_cg_params dummy{1e-10, 1, SM_F64, 0.1, SM_CG_AUTO};
  SM_TRY(force_at(c, q, c.w.U64, c.w.U32, phi, part, cg ? *cg : dummy, F, nullptr, 0.0,
                  part == SM_PART_HEAVY ? phi : nullptr));
  return c.sync();
}

int sm_fermion_force(const sm_lattice* lat, const double* q, const double* phi,
                     const sm_cg_params* cg, double* F, void* ws, size_t ws_bytes,
                     sm_stats* stats, void* stream) {
  return sm_force(lat, q, phi, SM_PART_FERMION, cg, F, ws, ws_bytes, stats, stream);
}

int sm_fg_shifted_force(const sm_lattice* lat, const double* q, const double* phi, int part,
                        double h, const sm_cg_params* cg, double* F, void* ws, size_t ws_bytes,
                        sm_stats* stats, void* stream) {
  Ctx c;
  SM_TRY(c.init(lat, ws, ws_bytes, stream, stats));
  SM_TRY(check_split_part(lat, part));
  SM_TRY(check_cg(cg));
  SM_TRY(fields_ok({q, F}, "sm_fg_shifted_force"));
  if (part & ~SM_PART_GAUGE) {
    SM_TRY(fields_ok({phi}, "sm_fg_shifted_force"));
    SM_TRY(make_links(c, q, c.w.U64, c.w.U32, *cg));
  }
  SM_TRY(shifted_force(c, q, c.w.U64, c.w.U32, phi, part, h, *cg, F, nullptr, 0.0,
                       part == SM_PART_HEAVY ? phi : nullptr));
  return c.sync();
}

int sm_force_gradient(const sm_lattice* lat, const double* q, const double* phi, int part,
                      const sm_cg_params* cg, double* C, double* F, void* ws, size_t ws_bytes,
                      sm_stats* stats, void* stream) {
  Ctx c;
  SM_TRY(c.init(lat, ws, ws_bytes, stream, stats));
  if (part == SM_PART_HEAVY)
    return fail(SM_ERR_ARG, "sm_force_gradient: no force-gradient term of the heavy part");
  SM_TRY(check_split_part(lat, part));
  SM_TRY(check_cg(cg));
  SM_TRY(fields_ok({q, C}, "sm_force_gradient"));
  if (F && !al16(F)) return fail(SM_ERR_ARG, "sm_force_gradient: F not aligned");
  if (part & ~SM_PART_GAUGE) {
    SM_TRY(fields_ok({phi}, "sm_force_gradient"));
    SM_TRY(make_links(c, q, c.w.U64, c.w.U32, *cg));
  }
  SM_TRY(force_and_gradient(c, q, c.w.U64, c.w.U32, phi, part, *cg, C));
  if (F) SM_CU(cudaMemcpyAsync(F, c.w.F, sizeof(double) * 2 * lat->N, cudaMemcpyDeviceToDevice, c.s));
  return c.sync();
}

int sm_hvp(const sm_lattice* lat, const double* q, const double* phi, int part, const double* v,
           const sm_cg_params* cg, double* Hv, void* ws, size_t ws_bytes, sm_stats* stats,
           void* stream) {
  Ctx c;
  SM_TRY(c.init(lat, ws, ws_bytes, stream, stats));
  SM_TRY(check_part(part));
  SM_TRY(check_cg(cg));
  SM_TRY(fields_ok({q, v, Hv}, "sm_hvp"));
  if (part & SM_PART_FERMION) {
    SM_TRY(fields_ok({phi}, "sm_hvp"));
    SM_TRY(make_links(c, q, c.w.U64, c.w.U32, *cg));
    SM_TRY(chi_xi(c, c.w.U64, c.w.U32, phi, *cg));
  }
  SM_TRY(launch_lincomb(c, c.w.v, nullptr, 1.0, v, 0.0, nullptr));
  SM_TRY(hess_times(c, q, c.w.U64, c.w.U32, part, c.w.v, *cg, Hv));
  SM_TRY(launch_lincomb(c, Hv, nullptr, 0.5, Hv, 0.0, nullptr));
  return c.sync();
}

int sm_energies(const sm_lattice* lat, const double* q, const double* p, const double* phi,
                const sm_cg_params* cg, double* K, double* S_G, double* S_F, void* ws,
                size_t ws_bytes, sm_stats* stats, void* stream) {
  Ctx c;
  SM_TRY(c.init(lat, ws, ws_bytes, stream, stats));
  if ((K && !p) || ((S_G || S_F) && !q)) return fail(SM_ERR_ARG, "sm_energies: missing field");
  if (S_F) {
    SM_TRY(check_cg(cg));
    SM_TRY(fields_ok({q, phi}, "sm_energies"));
    SM_TRY(make_links(c, q, c.w.U64, c.w.U32, *cg));
    SM_TRY(cg_solve(c, c.w.U64, c.w.U32, phi, c.w.xi, *cg, nullptr, nullptr));
  }
  SM_TRY(launch_energies(c, S_G ? q : nullptr, K ? p : nullptr, S_F ? phi : nullptr,
                         S_F ? c.w.xi : nullptr, K, S_G, S_F));
  return c.sync();
}

int sm_md_trajectory(const sm_lattice* lat, double* q, double* p, const double* phi,
                     const sm_md_params* md, void* ws, size_t ws_bytes, sm_stats* stats,
                     void* stream) {
  Ctx c;
  SM_TRY(c.init(lat, ws, ws_bytes, stream, stats));
  SM_TRY(check_md(md, lat));
  if (md->n < 1 || !(md->tau > 0)) return fail(SM_ERR_ARG, "md: n >= 1 and tau > 0 required");
  SM_TRY(fields_ok({q, p, phi}, "sm_md_trajectory"));
  c.strict = false;
  SM_TRY(md_run(c, q, p, phi, *md, md->tau / md->n, md->n));
  SM_TRY(c.sync());
  return chain_failures(c, "sm_md_trajectory");
}

int sm_md_step(const sm_lattice* lat, double* q, double* p, const double* phi,
               const sm_md_params* md, double h, void* ws, size_t ws_bytes, sm_stats* stats,
               void* stream) {
  Ctx c;
  SM_TRY(c.init(lat, ws, ws_bytes, stream, stats));
  SM_TRY(check_md(md, lat));
  SM_TRY(fields_ok({q, p, phi}, "sm_md_step"));
  c.strict = false;
  SM_TRY(md_run(c, q, p, phi, *md, h, 1));
  SM_TRY(c.sync());
  return chain_failures(c, "sm_md_step");
}

}  // extern "C"

namespace sm {

// S_h + S_r of the split action at the links in c.w.U64/U32 into Sr[nchains]
// (with the kinetic term and S_G when p, q are given) and Sh[nchains].
static int split_energies(Ctx& c, const double* q, const double* p, const sm_cg_params& cgH,
                          double* K, double* SG, double* Sr, double* Sh) {
  Ctx h = heavy_ctx(c);
  SM_TRY(launch_dslash<double>(h, c.w.U64, c.w.phi, c.w.psi, true, nullptr, 0.0));
  SM_TRY(cg_solve(c, c.w.U64, c.w.U32, c.w.psi, c.w.xi, cgH, nullptr, nullptr));
  SM_TRY(launch_energies(c, q, p, c.w.psi, c.w.xi, K, SG, Sr));
  const int rc = cg_solve(h, c.w.U64, c.w.U32, c.w.phi_h, c.w.xi, cgH, nullptr, nullptr);
  merge_flags(c, h);
  if (rc) return rc;
  return launch_energies(c, nullptr, nullptr, c.w.phi_h, c.w.xi, nullptr, nullptr, Sh);
}

// The device part of one HMC update of every chain (Sec. 2.1): heatbath
// phi = D^dag eta, H at the start, the MD trajectory, H at the end.  Enqueues
// only (no host synchronisation when c.deferred).  Energies land in
// c.w.out = [K0, SG0, SF0, K1, SG1, SF1, Sh0, Sh1][nchains]: SF the fermion
// action (the ratio part S_r for the three-level schemes), Sh the heavy part
// S_h (zero without the split).
static int hmc_enqueue(Ctx& c, double* q, const double* p0, const double* eta,
                       const sm_md_params& md) {
  const int nc = c.L->nchains;
  const size_t lbytes = sizeof(double) * 2 * (size_t)c.L->N;
  const sm_cg_params& cg = md.cg;
  sm_cg_params cgH = cg;  // the S_F solves of H
  if (md.tol_action > 0.0) cgH.tol = md.tol_action;
  double* out = c.w.out;
  Range range("hmc:trajectory");
  if (c.deferred) SM_CU(cudaMemsetAsync(c.w.acc, 0, 3 * sizeof(int) * nc, c.s));
  SM_TRY(make_links(c, q, c.w.U64, c.w.U32, cg));
  if (three_level(md.scheme)) {
    // phi_h = D_h^dag eta_h; phi_r = D_h^dag^{-1} D^dag eta_r = D_h (D_h^dag D_h)^{-1} D^dag eta_r
    const double* eta_r = eta;
    const double* eta_h = eta + 4 * (size_t)c.L->N;
    Ctx h = heavy_ctx(c);
    SM_TRY(launch_dslash<double>(h, c.w.U64, eta_h, c.w.phi_h, true, nullptr, 0.0));
    SM_TRY(launch_dslash<double>(c, c.w.U64, eta_r, c.w.b, true, nullptr, 0.0));
    bool have = false;
    int rc = cg_solve(h, c.w.U64, c.w.U32, c.w.b, c.w.xi, cg, nullptr, nullptr, c.w.phi, &have);
    merge_flags(c, h);
    if (rc) return rc;
    if (!have) SM_TRY(launch_dslash<double>(h, c.w.U64, c.w.xi, c.w.phi, false, nullptr, 0.0));
    SM_CU(cudaMemcpyAsync(c.w.qsave, q, lbytes, cudaMemcpyDeviceToDevice, c.s));
    SM_CU(cudaMemcpyAsync(c.w.pw, p0, lbytes, cudaMemcpyDeviceToDevice, c.s));
    if (md.sf_start == SM_SF_NOISE) {
      // S_r = eta_r^dag eta_r, S_h = eta_h^dag eta_h for the pseudofermions above
      SM_TRY(launch_energies(c, q, c.w.pw, eta_r, eta_r, out, out + nc, out + 2 * nc));
      SM_TRY(launch_energies(c, nullptr, nullptr, eta_h, eta_h, nullptr, nullptr, out + 6 * nc));
    } else {
      SM_TRY(split_energies(c, q, c.w.pw, cgH, out, out + nc, out + 2 * nc, out + 6 * nc));
    }
    SM_TRY(md_run(c, q, c.w.pw, c.w.phi, md, md.tau / md.n, md.n, c.w.phi_h));
    SM_TRY(make_links(c, q, c.w.U64, c.w.U32, cg));
    return split_energies(c, q, c.w.pw, cgH, out + 3 * nc, out + 4 * nc, out + 5 * nc,
                          out + 7 * nc);
  }
  SM_CU(cudaMemsetAsync(out + 6 * nc, 0, 2 * sizeof(double) * nc, c.s));
  SM_TRY(launch_dslash<double>(c, c.w.U64, eta, c.w.phi, true, nullptr, 0.0));
  SM_CU(cudaMemcpyAsync(c.w.qsave, q, lbytes, cudaMemcpyDeviceToDevice, c.s));
  SM_CU(cudaMemcpyAsync(c.w.pw, p0, lbytes, cudaMemcpyDeviceToDevice, c.s));
  if (md.sf_start == SM_SF_NOISE) {
    // S_F = phi^dag (D^dag D)^{-1} phi = eta^dag eta for phi = D^dag eta
    SM_TRY(launch_energies(c, q, c.w.pw, eta, eta, out, out + nc, out + 2 * nc));
  } else {
    SM_TRY(cg_solve(c, c.w.U64, c.w.U32, c.w.phi, c.w.xi, cgH, nullptr, nullptr));
    SM_TRY(launch_energies(c, q, c.w.pw, c.w.phi, c.w.xi, out, out + nc, out + 2 * nc));
  }
  SM_TRY(md_run(c, q, c.w.pw, c.w.phi, md, md.tau / md.n, md.n));
  SM_TRY(make_links(c, q, c.w.U64, c.w.U32, cg));
  SM_TRY(cg_solve(c, c.w.U64, c.w.U32, c.w.phi, c.w.xi, cgH, nullptr, nullptr));
  return launch_energies(c, q, c.w.pw, c.w.phi, c.w.xi, out + 3 * nc, out + 4 * nc, out + 5 * nc);
}

// Reads H (and, in deferred mode, the solves' flags), takes the Metropolis
// decisions and restores the links of rejected chains.  Synchronises.
static int hmc_finish(Ctx& c, double* q, const double* u, double* dH, double* H0, int* accepted,
                      double* p_out, double* q_md) {
  Range range("hmc:metropolis");
  const int nc = c.L->nchains;
  const size_t lbytes = sizeof(double) * 2 * (size_t)c.L->N;
  std::vector<double> h(8 * (size_t)nc);
  std::vector<int> acc(3 * (size_t)nc, 0);
  SM_CU(cudaMemcpyAsync(h.data(), c.w.out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c.s));
  if (c.deferred)
    SM_CU(cudaMemcpyAsync(acc.data(), c.w.acc, sizeof(int) * acc.size(), cudaMemcpyDeviceToHost, c.s));
  SM_CU(cudaStreamSynchronize(c.s));
  if (c.deferred) {
    c.chain_flags.assign(nc, 0);
    for (int i = 0; i < nc; ++i) {
      c.chain_flags[i] = acc[i];
      c.st->chain_iterations += acc[nc + i];
      c.st->reliable_updates += acc[2 * nc + i];
    }
    SM_TRY(profile_collect_deferred(c.L, acc.data() + nc));
  }
  // Metropolis: accept iff dH <= 0 or u < exp(-dH); non-finite dH rejects
  std::vector<int> reject(nc);
  bool any_nan = false, any_reject = false;
  for (int i = 0; i < nc; ++i) {
    const double h0 = h[i] + h[nc + i] + h[2 * nc + i] + h[6 * nc + i];
    const double h1 = h[3 * nc + i] + h[4 * nc + i] + h[5 * nc + i] + h[7 * nc + i];
    const double d = h1 - h0;
    dH[i] = d;
    if (H0) H0[i] = h0;
    const bool solved = c.chain_flags.empty() || c.chain_flags[i] == 0;
    const bool ok = solved && std::isfinite(d) && (d <= 0.0 || u[i] < std::exp(-d));
    accepted[i] = ok ? 1 : 0;
    reject[i] = ok ? 0 : 1;
    any_reject |= !ok;
    any_nan |= !std::isfinite(d);
  }
  if (p_out) SM_CU(cudaMemcpyAsync(p_out, c.w.pw, lbytes, cudaMemcpyDeviceToDevice, c.s));
  if (q_md) SM_CU(cudaMemcpyAsync(q_md, q, lbytes, cudaMemcpyDeviceToDevice, c.s));
  if (any_reject) {
    SM_CU(cudaMemcpyAsync(c.w.flags, reject.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, c.s));
    SM_TRY(launch_copy_links_masked(c, q, c.w.qsave, c.w.flags));
  }
  SM_TRY(c.sync());
  if (any_nan) return fail(SM_ERR_NAN, "hmc: non-finite Delta H (chain rejected)");
  return chain_failures(c, "hmc");
}

static bool all_chain_resident(const sm_lattice* L, const sm_md_params& md) {
  sm_cg_params cgH = md.cg;
  if (md.tol_action > 0.0) cgH.tol = md.tol_action;
  return chain_cg_selected(L, md.cg) && chain_cg_selected(L, cgH);
}

}  // namespace sm

// A captured HMC trajectory (see sm_hmc_graph_create).
struct sm_hmc_graph {
  const sm_lattice* lat;
  double* q;
  void* ws;
  size_t ws_bytes;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  long long kernels;  // kernel nodes: launches per replay
};

extern "C" {

int sm_hmc_trajectory(const sm_lattice* lat, double* q, const double* p0, const double* eta,
                      const double* u, const sm_md_params* md, void* ws, size_t ws_bytes,
                      double* dH, double* H0, int* accepted, double* p_out, double* q_md,
                      sm_stats* stats, void* stream) {
  Ctx c;
  SM_TRY(c.init(lat, ws, ws_bytes, stream, stats));
  SM_TRY(check_md(md, lat));
  if (md->n < 1 || !(md->tau > 0)) return fail(SM_ERR_ARG, "md: n >= 1 and tau > 0 required");
  SM_TRY(fields_ok({q, p0, eta}, "sm_hmc_trajectory"));
  if (!u || !dH || !accepted) return fail(SM_ERR_ARG, "sm_hmc_trajectory: NULL host output");
  if ((p_out && !al16(p_out)) || (q_md && !al16(q_md)))
    return fail(SM_ERR_ARG, "sm_hmc_trajectory: unaligned output");
  c.strict = false;  // a failing chain is rejected, the others go on
  c.deferred = all_chain_resident(lat, *md);
  SM_TRY(hmc_enqueue(c, q, p0, eta, *md));
  return hmc_finish(c, q, u, dH, H0, accepted, p_out, q_md);
}

int sm_hmc_graph_create(const sm_lattice* lat, double* q, const double* p0, const double* eta,
                        const sm_md_params* md, void* ws, size_t ws_bytes, sm_hmc_graph** out,
                        void* stream) {
  if (!out) return fail(SM_ERR_ARG, "sm_hmc_graph_create: out is NULL");
  *out = nullptr;
  if (!stream) return fail(SM_ERR_ARG, "sm_hmc_graph_create: needs a non-default stream");
  Ctx c;
  SM_TRY(c.init(lat, ws, ws_bytes, stream, nullptr));
  SM_TRY(check_md(md, lat));
  if (md->n < 1 || !(md->tau > 0)) return fail(SM_ERR_ARG, "md: n >= 1 and tau > 0 required");
  SM_TRY(fields_ok({q, p0, eta}, "sm_hmc_graph_create"));
  if (!all_chain_resident(lat, *md))
    return fail(SM_ERR_ARG, "sm_hmc_graph_create: every solve must be chain-resident "
                            "(SM_CG_AUTO or SM_CG_CHAIN with chains that fit)");
  SM_TRY(chain_cg_prepare(lat, md->cg));
  SM_TRY(c.sync());
  c.strict = false;
  c.deferred = true;
  c.capturing = true;
  const long long before = sm_launch_count();
  SM_CU(cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal));
  const int rc = hmc_enqueue(c, q, p0, eta, *md);
  const long long captured = sm_launch_count() - before;
  add_launches(-captured);  // captured launches run only when the graph is replayed
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c.s, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  cudaGraphExec_t x = nullptr;
  const cudaError_t e2 = cudaGraphInstantiate(&x, g, 0);
  if (e2 != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(SM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e2));
  }
  *out = new sm_hmc_graph{lat, q, ws, ws_bytes, g, x, captured};
  return SM_OK;
}

int sm_hmc_graph_run(sm_hmc_graph* gr, const double* u, double* dH, double* H0, int* accepted,
                     sm_stats* stats, void* stream) {
  if (!gr) return fail(SM_ERR_ARG, "sm_hmc_graph_run: graph is NULL");
  if (!u || !dH || !accepted) return fail(SM_ERR_ARG, "sm_hmc_graph_run: NULL host output");
  Ctx c;
  SM_TRY(c.init(gr->lat, gr->ws, gr->ws_bytes, stream, stats));
  c.strict = false;
  c.deferred = true;
  SM_CU(cudaGraphLaunch(gr->exec, c.s));
  add_launches(gr->kernels);
  c.st->kernel_launches += gr->kernels;
  return hmc_finish(c, gr->q, u, dH, H0, accepted, nullptr, nullptr);
}

int sm_hmc_graph_destroy(sm_hmc_graph* gr) {
  if (!gr) return SM_OK;
  if (gr->exec) cudaGraphExecDestroy(gr->exec);
  if (gr->graph) cudaGraphDestroy(gr->graph);
  delete gr;
  return SM_OK;
}

}  // extern "C"
