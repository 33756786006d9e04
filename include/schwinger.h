/*
 * schwinger.h -- C ABI of the GB300 (sm_103a) Schwinger-model HMC library.
 *
 * The library implements the molecular-dynamics hot path of Hybrid Monte
 * Carlo for the two-dimensional U(1) gauge theory with two degenerate Wilson
 * fermions (one pseudofermion), as set out in "Adapted nested force-gradient
 * integrators: the Schwinger model case" (arXiv:1512.03812):
 *   the Wilson-Dirac operator D and D^dag (Sec. 3, Wilson-Dirac matrix),
 *   conjugate-gradient solves of D^dag D x = phi (Sec. 3, Eq. fer_action,
 *   Eq. chi_xi_vectors), the gauge and fermion forces (Eq. force_gauge,
 *   Eq. force_fermion), the exact force-gradient term (Eq. force_gradient,
 *   Eq. CFF, Eq. Z12) and its shifted-force approximation (Sec. 2), the
 *   link and momentum updates (Sec. 2.1) and the integration schemes of
 *   Sec. 2 (Eq. leap ... Eq. ad_5stage_multi_fg), and the HMC trajectory
 *   with its Metropolis step (Sec. 2.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Batch.  A lattice object holds a batch of independent chains; chain c is an
 *   L_c x T_c lattice with its own beta_c and m0_c.  Chains may differ in size.
 *   Sites of all chains are stored back to back: chain c occupies global
 *   sites [off_c, off_c + L_c T_c), off_0 = 0, off_{c+1} = off_c + L_c T_c.
 *   Within a chain, site n = (x, t) has local index x + L_c t (x fastest).
 * Directions.  mu = 0 is x (the paper's mu = 1), mu = 1 is t (mu = 2).
 * Boundary conditions.  Gauge links are periodic; fermions are periodic in x
 *   and antiperiodic in t.
 * Layouts (all device memory, all owned by the caller):
 *   link angles q, momenta p, forces F, C, directions v:
 *       double [N][2]    (site-major, mu fastest), N = total sites
 *   links U64: double [N][2][2]  -- U_mu(n) as (Re, Im); the antiperiodic
 *       fermion sign is folded in: links U_t(x, T_c - 1) are stored negated.
 *   links U32: float  [N][2][2]  -- the same in FP32.
 *   spinors:  double [N][2][2] (FP64) or float [N][2][2] (FP32):
 *       per site two spin components, each (Re, Im).
 *   per-chain outputs (actions, Delta H, ...): double [nchains].
 *   Every pointer must be aligned to 16 bytes.
 * Streams.  `stream` is a cudaStream_t passed as void*; NULL is the legacy
 *   default stream.  Entry points enqueue work on it and return without
 *   synchronising, except where they return host-side results (marked
 *   "synchronises").
 * Workspace.  Entry points that need scratch take a device buffer `ws` of at
 *   least sm_workspace_bytes(lat) bytes (256-byte aligned) and allocate
 *   nothing themselves.  The contents of `ws` are not preserved between
 *   calls, and two calls that use one workspace must not overlap in time.
 * Errors.  Every entry point returns SM_OK (0) or an SM_ERR_* code and never
 *   throws.  sm_last_error() returns the calling thread's last message.
 *   After SM_ERR_CUDA the CUDA context may be unusable.
 */
#ifndef SCHWINGER_GB300_H
#define SCHWINGER_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SM_OK 0
#define SM_ERR_ARG 1            /* invalid argument (null, size, alignment) */
#define SM_ERR_CUDA 2           /* a CUDA call failed */
#define SM_ERR_NOT_CONVERGED 3  /* CG reached maxit for at least one chain */
#define SM_ERR_TIMEOUT 4        /* a bounded device-side wait expired */
#define SM_ERR_NAN 5            /* a non-finite value (e.g. Delta H) */

/* arithmetic of a field or a solve */
#define SM_F64 0    /* FP64 fields and FP64 CG */
#define SM_F32 1    /* FP32 fields (apply_D / apply_DdagD only) */
#define SM_MIXED 2  /* CG with FP32 iterations and FP64 reliable updates */

/* which part of the action S = S_G + S_F (Eq. schwinger) */
#define SM_PART_GAUGE 1
#define SM_PART_FERMION 2
#define SM_PART_FULL 3
/* With the fermion determinant split over two masses (sm_lattice_set_heavy;
 * the factorisation the paper's Conclusions call for, in the form of
 * Hasenbusch's mass split): det(D^dag D) = det(D_h^dag D_h) det(W^dag W),
 * W = D D_h^{-1}, D_h the Wilson-Dirac operator at the bare mass m0 + dm,
 *   S_h = phi_h^dag (D_h^dag D_h)^{-1} phi_h                (heavy part)
 *   S_r = phi_r^dag D_h (D^dag D)^{-1} D_h^dag phi_r        (ratio part). */
#define SM_PART_HEAVY 4
#define SM_PART_RATIO 8

/* integration schemes of Sec. 2 */
#define SM_LEAPFROG 0            /* Eq. leap */
#define SM_FIVE_STAGE 1          /* Eq. 5stage (weight lambda; 1/6 as printed) */
#define SM_FIVE_STAGE_FG 2       /* Eq. 5stage_fg, full C */
#define SM_NESTED_LEAPFROG 3     /* Eq. leap_multi */
#define SM_NESTED_FIVE_STAGE 4   /* Eq. 5stage_multi */
#define SM_NESTED_FG 5           /* Eq. 5stage_multi_fg (C_FF outside, C_GG inside) */
#define SM_ADAPTED_NESTED_FG 6   /* Eq. ad_5stage_multi_fg (C_FF outside, leapfrog inside) */
#define SM_ELEVEN_STAGE 7        /* Eq. 11_stage, with the weights of Eq. (71) of Omelyan,
                                    Mryglod and Folk (2003) that the paper cites */
/* Three time scales on the determinant split over two masses (the paper's
 * Conclusions: more than two parts, force-gradient information only for the
 * most expensive one, leapfrog for the fast ones).  B3 = S_r outside, B2 =
 * S_h in the middle (md.M2 leapfrog steps per middle block), B1 = S_G inside
 * (md.M leapfrog steps per gauge block). */
#define SM_NESTED3_LEAPFROG 8    /* Eq. leap_multi on three levels */
#define SM_ADAPTED_NESTED3_FG 9  /* Eq. ad_5stage_multi_fg with S_r outside and C of S_r
                                    alone, leapfrog levels of S_h and S_G inside */

/* how a force-gradient kick obtains C */
#define SM_FG_EXACT 0    /* exact C via one extra CG (Eq. CFF, Eq. Z12) */
#define SM_FG_SHIFTED 1  /* force at the shifted field q - (h^2/24) F(q) (Sec. 2) */

typedef struct sm_lattice sm_lattice;

/* S_F at the start of a trajectory (sm_md_params.sf_start) */
#define SM_SF_SOLVE 0
#define SM_SF_NOISE 1

/* how a batched CG solve is laid out on the GPU */
#define SM_CG_AUTO 0   /* chain-resident when every chain fits, else grid-wide */
#define SM_CG_GRID 1   /* all chains advance together, two launches per iteration */
#define SM_CG_CHAIN 2  /* one thread block owns one chain's whole solve; FP32 fields in
                          shared memory (chains of at most 4096 sites for SM_MIXED,
                          16384 for SM_F64) */
#define SM_CG_VARIANTS 9  /* kernel variants of the chain-resident mixed CG (sm_autotune_cg) */

/* CG parameters.  The solve of D^dag D x = b starts from x = 0 and stops, per
 * chain, when |b - D^dag D x| <= tol |b|: for SM_F64 the recursive residual
 * is tested, for SM_MIXED the FP64 true residual recomputed at each reliable
 * update.  A reliable update is taken when the FP32 residual has fallen by
 * the factor `delta` (0 < delta < 1) below its largest value since the last
 * one.  In the chain-resident column-pair kernels an update that only
 * restarts the FP32 recurrence computes the residual in double-float
 * arithmetic (float pairs, about 48 bits); a solve ends only on an FP64
 * update, whose true residual is the one tested.  maxit bounds the
 * iterations of every chain. */
typedef struct {
  double tol;
  int maxit;
  int prec;      /* SM_F64 or SM_MIXED */
  double delta;  /* reliable-update factor, e.g. 0.1 (SM_MIXED only) */
  int algo;      /* SM_CG_AUTO, SM_CG_GRID or SM_CG_CHAIN */
} sm_cg_params;

/* One molecular-dynamics trajectory: n steps of size h = tau / n of `scheme`;
 * M inner steps per inner block for the nested schemes; `lambda` the outer
 * weight of the five-stage schemes (1/6 in Eq. 5stage; 0.1931833275 for
 * Omelyan's minimum-norm variant); `fg` one of SM_FG_*.  With merge_kicks != 0
 * adjacent kicks of the same action part are applied as one kick (the same
 * flow, fewer force evaluations). */
typedef struct {
  int scheme;
  double tau;
  int n;
  int M;
  double lambda;
  int fg;
  int merge_kicks;
  sm_cg_params cg;
  double tol_action;  /* CG tolerance of the S_F solves of H in sm_hmc_trajectory
                         (0: cg.tol); the MD force solves use cg.tol */
  int sf_start;       /* S_F in H at the start of sm_hmc_trajectory: SM_SF_SOLVE (a CG
                         solve, like the end) or SM_SF_NOISE (eta^dag eta, exact for
                         phi = D^dag eta; one solve fewer) */
  int M2;             /* three-level schemes: leapfrog steps of the heavy part per middle
                         block (>= 1; ignored by the other schemes) */
} sm_md_params;

/* Counters accumulated over one call (zeroed by the call). */
typedef struct {
  long long cg_solves;         /* batched CG solves of D^dag D */
  long long cg_iterations;     /* batched iterations (all chains advance together) */
  long long chain_iterations;  /* sum over chains of their own iteration counts */
  long long reliable_updates;  /* FP64 reliable updates, summed over chains */
  long long inversions;        /* inversions of D in the paper's units (Sec. 3, end) */
  long long force_evals;       /* fermion-force evaluations */
  long long kernel_launches;   /* device kernels launched by this call */
} sm_stats;

/* ------------------------------------------------------------ library ---- */

/* Thread-local description of the last error (never NULL). */
const char* sm_last_error(void);
/* ABI version: 1. */
int sm_version(void);
/* Total device kernels launched by this library in this process. */
long long sm_launch_count(void);

/* Kernel timing of the CG iterations, for roofline reporting.  While enabled,
 * every chunk of batched CG iterations (the two kernels of an iteration,
 * repeated) and every FP64 residual pass is bracketed by CUDA events on the
 * solve's stream.  sm_profile_read returns the accumulated device time of the
 * iteration kernels (iter_ms) and of the FP64 residual passes (res_ms), the
 * number of batched iterations launched, and the number of site-iterations
 * that did work (sum over chains of iterations x sites); reset != 0 zeroes
 * the accumulators.  Not thread-safe; for one device. */
int sm_profile_enable(int on);
int sm_profile_read(double* iter_ms, double* res_ms, long long* batched_iters,
                    long long* site_iters, int reset);

/* ----------------------------------------------------- lattice objects ---- */

/* Creates a batch of `nchains` >= 1 chains with sides L[c], T[c] >= 2 and
 * couplings beta[c] (Eq. gauge_action) and m0[c] (bare mass of the
 * Wilson-Dirac operator; kappa = 1 / (2 (2 + m0))).  Host arrays, copied.
 * Allocates the geometry tables on the current device.  Returns
 * SM_ERR_ARG on a bad size and SM_ERR_CUDA on an allocation failure. */
int sm_lattice_create(int nchains, const int* L, const int* T, const double* beta,
                      const double* m0, sm_lattice** out);
int sm_lattice_destroy(sm_lattice* lat);
/* Splits the fermion determinant of every chain over the masses m0_c and
 * m0_c + dm (SM_PART_HEAVY, SM_PART_RATIO, the three-level schemes): keeps a
 * second copy of the lattice's tables at the heavy masses (allocates; call
 * it at set-up, and size workspaces with sm_workspace_bytes afterwards: the
 * split needs two more spinor fields).  dm > 0; calling it again changes dm.
 * Then:
 *   sm_force / sm_fermion_force-like calls with part SM_PART_HEAVY take phi =
 *     phi_h, with SM_PART_RATIO phi = phi_r (one part per call);
 *   sm_force_gradient with SM_PART_RATIO returns C of S_r alone;
 *   sm_md_trajectory / sm_md_step with a three-level scheme take phi =
 *     [phi_r; phi_h] (2N spinors, phi_r first);
 *   sm_hmc_trajectory / sm_hmc_graph_create with a three-level scheme take
 *     eta = [eta_r; eta_h] (2N spinors): phi_h = D_h^dag eta_h and
 *     phi_r = D_h^dag^{-1} D^dag eta_r, so that S_h = eta_h^dag eta_h and
 *     S_r = eta_r^dag eta_r at the start; H = K + S_G + S_h + S_r.
 * SM_ERR_ARG if dm <= 0 or not finite, SM_ERR_CUDA on an allocation failure. */
int sm_lattice_set_heavy(sm_lattice* lat, double dm);

/* Reads and clears the lattice's device error word after synchronising the
 * device: nonzero (and SM_ERR_TIMEOUT) if a bounded device-side wait of a
 * kernel on this lattice gave up since the last check (for example a TMA copy
 * that did not complete; the affected tile was not computed). */
int sm_lattice_check(const sm_lattice* lat, int* code);
/* Bounds checks of the debug build (the library compiled with -DSM_DEBUG):
 * reads and clears the count of out-of-range indices met since the last
 * read, with the first such index and the code of the place it came from
 * (1: a site index of a field access, checked against the site count of the
 * call's lattice; 10-14: a neighbour of the chain-resident CG's shared-memory
 * layout; 20-29: a halo index of the tiled D^dag D).  In the debug build an
 * out-of-range access is redirected to index 0 instead of being made, so a
 * kernel with an indexing error runs to its end and the error is reported
 * here.  Synchronises the device.  In the normal build the checks are not
 * compiled in: *violations = 0 and *first_where = -2.  No counterpart in the
 * paper: a substitute for a memory checker, for tests.  Host pointers;
 * SM_ERR_ARG if one is NULL. */
int sm_debug_read(long long* violations, long long* first_index, int* first_where);

/* Bound of a thread block's first wait for its TMA box copies (the interior
 * tiles of the fused D^dag D on single-chain lattices of at least 2^18 sites
 * too narrow for the streaming form, in sm_apply_DdagD and the grid-wide CG):
 * `polls` polls of the copies' mbarrier, 0 <= polls <= 4194304 (the
 * default); -1 restores the default.  A block whose first wait runs out
 * records SM_ERR_TIMEOUT in the lattice's error word (sm_lattice_check),
 * waits again, with the full bound, for its copies to land, and leaves its
 * tile uncomputed instead of waiting on.  No counterpart in the paper: a
 * control of the library's failure detection, so that a test can make the
 * wait run out (polls = 0: every such wait gives up at once) and check that
 * the error is reported and the context stays usable.  SM_ERR_ARG on a
 * NULL lattice or a value out of range. */
int sm_set_wait_limit(sm_lattice* lat, int polls);
/* Total number of sites N of the batch. */
long long sm_lattice_sites(const sm_lattice* lat);
int sm_lattice_chains(const sm_lattice* lat);
/* Bytes of workspace the entry points below require for this lattice. */
size_t sm_workspace_bytes(const sm_lattice* lat);

/* ------------------------------------------------------- field set-up ---- */

/* U_mu(n) = exp(i q_mu(n)) (Sec. 3, after Eq. gauge_action), with the
 * antiperiodic fermion sign folded into the t-links on the last time slice.
 * Writes U64 (may be NULL) and U32 (may be NULL). */
int sm_links(const sm_lattice* lat, const double* q, double* U64, float* U32, void* stream);

/* --------------------------------------------------- Wilson-Dirac D ------- */

/* out = D in (dagger = 0) or D^dag in (dagger = 1), the Wilson-Dirac
 * operator of Sec. 3:
 *   (D psi)(n) = (2 + m0) psi(n) - 1/2 sum_mu [ (1 - sigma_mu) U_mu(n) psi(n+mu)
 *                                  + (1 + sigma_mu) U_mu^dag(n-mu) psi(n-mu) ].
 * prec = SM_F64: U, in, out are FP64 (U = U64); SM_F32: all FP32 (U = U32).
 * `in` and `out` must not overlap. */
int sm_apply_D(const sm_lattice* lat, const void* U, const void* in, void* out, int dagger,
               int prec, void* stream);

/* out = D^dag D in (Eq. fer_action), same conventions as sm_apply_D, in one
 * fused pass (D in is kept on chip per tile).  ws is not used (may be NULL). */
int sm_apply_DdagD(const sm_lattice* lat, const void* U, const void* in, void* out, int prec,
                   void* ws, size_t ws_bytes, void* stream);

/* out = D^dag D in for ONE L x T lattice (sides >= 2, periodic x,
 * antiperiodic t, bare mass m0), without allocating anything.  The paper has
 * no counterpart: this is a service for callers that cannot call cudaMalloc
 * -- code whose device memory is all owned by a host framework's pool, code
 * that must not risk the device-wide synchronisation of an allocation, or
 * plugins that may not create allocations -- and therefore can create neither
 * a workspace nor a lattice object (sm_lattice_create allocates).
 * U, in, out as for sm_apply_D (prec SM_F64 or SM_F32, sites n = x + L t,
 * U with the antiperiodic sign folded in as written by sm_links); in and out
 * must not overlap.  The intermediate D in is kept in a built-in device array
 * of 8 MiB: at most 262144 sites in FP64 or 524288 in FP32; larger lattices
 * are rejected with SM_ERR_ARG.  The array is loaded with the library on
 * every GPU that uses it and held until the process exits.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current, and so does the first call after the device's context
 * was torn down and recreated (for example by cudaDeviceReset: the address is
 * cached with the context's unique id); make such a call before any stream
 * capture.  All
 * calls share the one array and each overwrites it completely before reading
 * it, so nothing carries over between calls -- but calls whose work can
 * overlap on the GPU (different streams, or concurrent host threads) race on
 * it and must be serialised by the caller.  Enqueues on `stream`, returns
 * without synchronising. */
int sm_apply_DdagD_noalloc(int L, int T, double m0, const void* U, const void* in, void* out,
                           int prec, void* stream);

/* Autotuner of the strip height of the streaming FP32 D^dag D (the form
 * sm_apply_DdagD takes for batches of at least 2^18 sites whose chains are
 * all wide enough: each warp walks a strip of 60 columns and `height` rows).
 * Times, on the given operands (U32, in, out as for sm_apply_DdagD with
 * SM_F32; out is overwritten), 10 launches back to back per candidate
 * height -- the lowest heights whose blocks fit on the GPU in 1, 2, 3 and 4
 * waves, and two and four times the one-wave height -- and keeps the fastest
 * in the lattice object for later sm_apply_DdagD calls.  The one-wave height
 * is the default before tuning.  height (host, may be NULL) receives the
 * choice (0 if the streaming form does not serve this lattice: then nothing
 * is timed), heights and ms (host [SM_DDAGD_HEIGHTS], may be NULL) each
 * candidate and its time per launch, -1 past the last.  No counterpart in
 * the paper: a tuning of the library's own tiling.  Allocates and frees the
 * candidates' strip tables (a set-up call, not for the hot path);
 * synchronises. */
#define SM_DDAGD_HEIGHTS 8
int sm_autotune_ddagd(sm_lattice* lat, const float* U32, const float* in, float* out,
                      int* height, int* heights, double* ms, void* stream);

/* -------------------------------------------------------- inversion ------- */

/* Solves D^dag D x = b for every chain (Sec. 3: the inversions behind
 * Eq. chi_xi_vectors; the solver is CG, see sm_cg_params).  U64 is always
 * needed; U32 is needed for SM_MIXED and may be NULL for SM_F64.  b, x FP64
 * spinors.  iters and relres (host arrays [nchains], may be NULL) receive
 * each chain's iteration count and final FP64 true relative residual.
 * Synchronises.  Returns SM_ERR_NOT_CONVERGED if a chain reached maxit
 * (x then holds its last iterate). */
int sm_cg_solve(const sm_lattice* lat, const double* U64, const float* U32, const double* b,
                double* x, const sm_cg_params* cg, void* ws, size_t ws_bytes, int* iters,
                double* relres, void* stream);

/* Autotuner of the chain-resident mixed-precision CG: times every kernel
 * variant that applies to this lattice's chain shapes (0: strided layout,
 * any chain up to 4096 sites; 1: column layout, 512 threads x 8 rows; 2:
 * column layout, 256 threads x 16 rows; 3: column layout split over a
 * cluster of two blocks, 256 threads x 8 rows each, rows exchanged through
 * distributed shared memory; 4: the same with 512 threads x 4 rows, one
 * block per SM; 5: column pairs, 512 threads x 2 columns x 4 rows of 64 x 64
 * chains; 6: column pairs, 256 threads x 2 columns x 8 rows; 7: column pairs
 * split over a cluster of two blocks, 128 threads x 2 columns x 8 rows each;
 * 8: variant 6 with the FP32 iterate x, each thread's own p between
 * iterations and its own links in tensor memory (TMEM, 512 columns per
 * block, allocated and freed by the kernel) and, in the registers x leaves free, each thread's own p through
 * the D walk and own t = D p through the D^dag walk; the arithmetic of 6 in
 * the same order)
 * on the given solve (b, FP64; x is overwritten), and stores the fastest in the
 * lattice object, which later SM_MIXED chain-resident solves use.  variant
 * (host, may be NULL) receives the choice, ms (host [SM_CG_VARIANTS], may be
 * NULL) each variant's time or -1 where it does not apply.  The variants differ only in their reduction order: results
 * agree to rounding, and a lattice object gives reproducible results once
 * tuned.  Needs SM_MIXED and chains of at most 4096 sites.  Synchronises. */
int sm_autotune_cg(sm_lattice* lat, const double* U64, const float* U32, const double* b,
                   double* x, const sm_cg_params* cg, void* ws, size_t ws_bytes, int* variant,
                   double* ms, void* stream);

/* Pins the kernel variant of the chain-resident mixed CG (as numbered for
 * sm_autotune_cg; -1 restores the default).  SM_ERR_ARG if it does not fit. */
int sm_set_cg_variant(sm_lattice* lat, int variant);

/* ----------------------------------------------------------- forces ------- */

/* F = dS_G/dq = beta g (Eq. force_gauge): F(n,x) = beta [sin th(n) - sin th(n-t)],
 * F(n,t) = beta [sin th(n-x) - sin th(n)], th(n) the plaquette angle. */
int sm_gauge_force(const sm_lattice* lat, const double* q, double* F, void* stream);

/* F = dS_F/dq = f (Eq. force_fermion) with chi, xi of Eq. chi_xi_vectors for
 * the pseudofermion phi (FP64 spinor).  One CG solve.  Synchronises. */
int sm_fermion_force(const sm_lattice* lat, const double* q, const double* phi,
                     const sm_cg_params* cg, double* F, void* ws, size_t ws_bytes,
                     sm_stats* stats, void* stream);

/* F = dS/dq for `part` (Eq. force).  Synchronises if part includes fermions. */
int sm_force(const sm_lattice* lat, const double* q, const double* phi, int part,
             const sm_cg_params* cg, double* F, void* ws, size_t ws_bytes, sm_stats* stats,
             void* stream);

/* F~ = F(q - (h^2/24) F(q)) for `part`: the shifted-field force whose Taylor
 * expansion F - (h^2/48) C supplies the force-gradient kick without C
 * (Sec. 2, the approximation after Eq. 5stage_fg).  Synchronises. */
int sm_fg_shifted_force(const sm_lattice* lat, const double* q, const double* phi, int part,
                        double h, const sm_cg_params* cg, double* F, void* ws,
                        size_t ws_bytes, sm_stats* stats, void* stream);

/* The exact force-gradient term C (Eq. force_gradient) for `part`:
 * SM_PART_GAUGE -> C_GG, SM_PART_FERMION -> C_FF, SM_PART_FULL ->
 * C_GG + C_FG + C_GF + C_FF (Eq. force_grad_de).  The fermion parts use the
 * sum-before-invert vectors Z_1, Z_2 of Eq. Z12, obtained from one CG solve.
 * F (may be NULL) receives the force of the same part.  Synchronises. */
int sm_force_gradient(const sm_lattice* lat, const double* q, const double* phi, int part,
                      const sm_cg_params* cg, double* C, double* F, void* ws,
                      size_t ws_bytes, sm_stats* stats, void* stream);

/* Hessian-vector product Hv = (d^2 S / dq dq) v for `part`: the second
 * derivative of Sec. 3.1 contracted with an arbitrary link field v (Eq. CFF
 * and Eq. Z12 with f replaced by v give 2 Hv for the fermion part).
 * Two CG solves for the fermion part.  Synchronises. */
int sm_hvp(const sm_lattice* lat, const double* q, const double* phi, int part,
           const double* v, const sm_cg_params* cg, double* Hv, void* ws, size_t ws_bytes,
           sm_stats* stats, void* stream);

/* Per-chain actions (device arrays [nchains]; each may be NULL):
 * S_G = beta sum (1 - Re P) (Eq. gauge_action), S_F = phi^dag (D^dag D)^{-1} phi
 * (Eq. fer_action; phi may be NULL when S_F is NULL) and the kinetic term
 * 1/2 sum p^2 (Eq. schwinger; p may be NULL when K is NULL).  FP64 sums in a
 * fixed order.  Synchronises if S_F is requested. */
int sm_energies(const sm_lattice* lat, const double* q, const double* p, const double* phi,
                const sm_cg_params* cg, double* K, double* S_G, double* S_F, void* ws,
                size_t ws_bytes, sm_stats* stats, void* stream);

/* --------------------------------------------------- integration ---------- */

/* Runs one MD trajectory (md->n steps of md->scheme, Sec. 2) in place on the
 * links q and momenta p of every chain, with pseudofermion phi.
 * Synchronises. */
int sm_md_trajectory(const sm_lattice* lat, double* q, double* p, const double* phi,
                     const sm_md_params* md, void* ws, size_t ws_bytes, sm_stats* stats,
                     void* stream);

/* One step of size h of md->scheme (md->tau and md->n are ignored). */
int sm_md_step(const sm_lattice* lat, double* q, double* p, const double* phi,
               const sm_md_params* md, double h, void* ws, size_t ws_bytes, sm_stats* stats,
               void* stream);

/* One HMC update of every chain (Sec. 2.1).  Inputs: links q (device, in/out),
 * momenta p0 and Gaussian noise eta (device, read only), Metropolis uniforms
 * u[nchains] in [0, 1) (host).  The pseudofermion is phi = D^dag eta at the
 * starting links; H = 1/2 sum p^2 + S_G + S_F (Eq. schwinger) is summed in FP64
 * before and after the trajectory; chain c is accepted iff
 * Delta H_c <= 0 or u[c] < exp(-Delta H_c), and a rejected (or non-finite)
 * chain gets its starting links back.  dH and H0 (host [nchains], H0 may be
 * NULL) receive Delta H and H at the start, accepted (host [nchains]) 1 or 0.
 * If p_out (device, may be NULL) is given it receives the momenta at the end
 * of the trajectory and q_md (device, may be NULL) the links before the
 * Metropolis step.  Synchronises. */
int sm_hmc_trajectory(const sm_lattice* lat, double* q, const double* p0, const double* eta,
                      const double* u, const sm_md_params* md, void* ws, size_t ws_bytes,
                      double* dH, double* H0, int* accepted, double* p_out, double* q_md,
                      sm_stats* stats, void* stream);

/* ------------------------------------------------ captured trajectories ---- */

/* One HMC update of every chain captured as a CUDA graph (Sec. 2.1, the same
 * computation as sm_hmc_trajectory): the device part -- heatbath, H at the
 * start, the MD trajectory, H at the end -- is recorded once on `stream` (a
 * non-default stream) and replayed by sm_hmc_graph_run; the Metropolis
 * decisions and the restoring of rejected chains follow each replay on the
 * host.  The graph is bound to the buffers given here: q (device, updated in
 * place by every run), p0 and eta (device; refill them between runs), ws,
 * and to md.  Every CG solve must be chain-resident (SM_CG_AUTO or
 * SM_CG_CHAIN, chains that fit): their per-chain outcomes stay on the device
 * until the end of a run.  Capture runs nothing.  The buffers and the lattice
 * must outlive the graph, and runs on one graph (or anything else using its
 * workspace) must not overlap.  The graph keeps the CG kernel variant the
 * lattice had when it was captured (tune with sm_autotune_cg first).  CG
 * kernel timing (sm_profile_enable) does not see solves inside a graph. */
typedef struct sm_hmc_graph sm_hmc_graph;
int sm_hmc_graph_create(const sm_lattice* lat, double* q, const double* p0, const double* eta,
                        const sm_md_params* md, void* ws, size_t ws_bytes, sm_hmc_graph** out,
                        void* stream);
/* Replays the captured trajectory and takes the Metropolis decisions as
 * sm_hmc_trajectory does (u, dH, H0, accepted host arrays [nchains]).
 * Synchronises. */
int sm_hmc_graph_run(sm_hmc_graph* g, const double* u, double* dH, double* H0, int* accepted,
                     sm_stats* stats, void* stream);
int sm_hmc_graph_destroy(sm_hmc_graph* g);

/* ------------------------------------------------- measured GPU rates ---- */

/* Micro-benchmarks of the rates the library's kernels are measured against
 * (no counterpart in the paper: they calibrate rooflines on the device in
 * use).  Each allocates and frees its own device memory, runs on the current
 * device's default stream, synchronises, and returns SM_OK or SM_ERR_CUDA.
 *
 * sm_peak_fma: dense fused multiply-add throughput in TFLOP/s (2 flops per
 *   FMA) of the FP64 (prec = SM_F64) or FP32 (SM_F32) pipes, from independent
 *   FMA chains in every thread of a grid filling all SMs.
 * sm_peak_l2_read: read bandwidth in GB/s of a `bytes`-sized buffer (at most
 *   the L2 size for an L2 figure) read `passes` times after one warm pass.
 * sm_peak_smem_read: shared-memory read bandwidth in GB/s over all SMs
 *   (16-byte loads by every thread of resident blocks). */
int sm_peak_fma(int prec, double* tflops);
int sm_peak_l2_read(long long bytes, int passes, double* gbs);
int sm_peak_smem_read(double* gbs);

#ifdef __cplusplus
}
#endif
#endif /* SCHWINGER_GB300_H */
