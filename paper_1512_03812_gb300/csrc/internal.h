// internal.h -- host-side declarations shared by the library's translation
// units: the lattice object, workspace carving, error reporting and the
// kernel launchers.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"
#include "schwinger.h"

struct sm_lattice {
  int nchains;
  long long N;
  int nblocks;
  std::vector<sm::ChainInfo> chains;
  sm::ChainInfo* d_chains;
  int* d_blk_chain;
  int* d_chain_list;  // [nchains] 0, 1, ..., nchains - 1
  int4* d_tiles;      // tiles of the fused D^dag D kernel (ddagd.cu)
  int ntiles;
  int4* d_tiles_big;  // 64 x 16 tiles of its large-lattice FP32 form
  int ntiles_big;
  // streaming FP32 D^dag D (stream.cuh): kSWarps strips {chain, xs, ts, dir}
  // per block ({chain, 0, 0, 0} pads a chain's last block), strips of
  // stream_tt rows; stream_ok if every chain is wide enough for it.  The
  // fused CG iteration has its own table (strips of stream_tt_cg rows;
  // ChainInfo::sb0, nsb index its blocks).
  bool stream_ok;
  int stream_tt, stream_tt_cg;
  int nstream, nstream_cg;  // blocks
  int4* d_stream;
  int4* d_stream_cg;
  int cg_variant;     // chain-resident mixed CG kernel chosen by sm_autotune_cg (-1: default)
  // mixed batches: chains of at most 4096 sites (solved chain-resident on the
  // side stream) and the mask of the others (solved grid-wide)
  int nsmall;
  int* d_small_list;
  int nbig;           // chains of the 4-block cluster shape (128 x 128), and their list
  int* d_big_list;
  // the chains of at most 4096 sites grouped by the kernel that serves their
  // shape (chain_group_kind): group g is d_group_list[group_begin[g] ..
  // group_begin[g] + group_count[g]); a mixed chain-resident solve of these
  // chains is one launch per group, the first group on the caller's stream,
  // the others on streams of their own
  static constexpr int kGroups = 5;
  int ngroups;
  int group_kind[kGroups], group_begin[kGroups], group_count[kGroups], group_vmax[kGroups];
  int* d_group_list;
  cudaStream_t gstream[kGroups];
  cudaEvent_t gev_fork, gev_join[kGroups];
  int nsm;            // multiprocessors of the device
  // the fermion determinant split over two masses (sm_lattice_set_heavy):
  // the same chains at the bare masses m0 + heavy_dm, or NULL
  sm_lattice* heavy;
  double heavy_dm;
  unsigned char* d_grid_mask;
  std::vector<unsigned char> grid_mask;
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  int* d_err;  // device-side error word (a bounded wait that gave up)
  int tma_spin;  // polls of the first wait for a tile's TMA box copies (sm_set_wait_limit)
  int device;
  int* h_pinned;  // small pinned host buffer for per-call readbacks
  cudaEvent_t ev[2];  // readback events of the CG loop
};

namespace sm {

// An NVTX range over the object's lifetime: visible to Nsight tools (and to
// ncu --nvtx-include), a cheap no-op without one.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Sets the thread-local message and returns `code`.
int fail(int code, const char* fmt, ...);
// Counts one kernel launch and checks the launch for errors.
int launched(sm_stats* st, const char* what);
// Adjusts the process-wide launch count (CUDA-graph capture and replay).
void add_launches(long long n);

// Per-chain CG scalars (device).
struct CgChain {
  double bb;       // |b|^2
  double rr;       // |r|^2 of the iterated residual
  double rr_prev;  // |r|^2 before the last iteration
  double alpha, beta;
  double rmax;     // largest |r|^2 since the last reliable update
  double rr_true;  // |b - A x|^2 at the last FP64 recomputation
  int state;       // 0 done, 1 iterating, 2 waiting for a reliable update
  int need_update; // reliable update requested
  int iters;
  int flags;       // bit 0: maxit reached, bit 1: breakdown (p^dag A p <= 0)
  int par;         // which of the two search-direction buffers holds p
  int updates;     // grid-wide form: reliable updates done
  double alpha_x;  // fused tiled form: x += alpha_x p still to be applied
};

// Scratch carved from the caller's workspace.
struct Ws {
  // FP64 spinors [N][2][2]
  double *r, *t, *p0, *p1, *xi, *chi, *s1, *s2, *z1, *z2, *phi, *b;
  // FP32 spinors
  float *r32, *x32, *p32a, *p32b, *t32;
  // links
  double *U64, *U64s;
  float *U32, *U32s;
  // real link fields [N][2]
  double *F, *C, *F2, *qs, *qsave, *pw, *v;
  double* sinp;  // [N] sine of the plaquette angle (gauge kick)
  // the split over two masses (lattices with a heavy copy only, carved after
  // everything else, so that the heavy copy's own carve of the same buffer
  // leaves them alone): the heavy pseudofermion and psi = D_h^dag phi_r
  double *phi_h, *psi;
  // reductions
  double* partials;    // [4][nblocks]
  unsigned* counters;  // [nchains]
  CgChain* cgc;        // [nchains]
  double* out;         // [8][nchains]
  int* flags;          // [nchains] per-chain masks
  int* acc;            // [3][nchains] accumulated CG flags, iterations, reliable updates (deferred)
  int* n_active;       // [2]: chains still iterating, chains due a reliable update
  int* order;          // [nchains] chains, longest previous solve first
  int* h_n_active;     // not in ws: pinned host word (see Ctx)

  static size_t bytes(const sm_lattice* L);
  int carve(const sm_lattice* L, void* ws, size_t nbytes);
};

// The per-call context: lattice, workspace, stream and counters.
struct Ctx {
  const sm_lattice* L;
  Geo g;
  Ws w;
  cudaStream_t s;
  sm_stats* st;
  sm_stats local;
  // Inside trajectories a chain whose solve fails (maxit, breakdown) must not
  // stop the others: with strict == false cg_solve ORs the chain's flags
  // into chain_flags and returns SM_OK.
  bool strict = true;
  std::vector<int> chain_flags;
  // Deferred mode (trajectories whose solves are all chain-resident, and
  // CUDA-graph capture): cg_solve does not read its results back; each
  // chain's flags and iteration count are accumulated on the device in
  // w.acc and read once at the end.
  bool deferred = false;
  bool capturing = false;  // inside a CUDA-graph capture (no profiling events)

  // ws_required: the entry point takes a workspace (then ws may not be NULL)
  int init(const sm_lattice* lat, void* ws, size_t nbytes, void* stream, sm_stats* stats,
           bool ws_required = true);
  dim3 grid() const { return dim3((unsigned)L->nblocks); }
  int zero_counters();
  int sync();
  int read_n_active(int* n);
};

// ------------------------------------------------------------ launchers ----
// All enqueue on c.s; R = double or float.
template <typename R>
int launch_dslash(Ctx& c, const R* U, const R* in, R* out, bool dagger, const R* add,
                  double add_scale);
int launch_links(Ctx& c, const double* q, double* U64, float* U32);
int launch_gauge_kick(Ctx& c, const double* q, double* p, double eps, double* Fout, bool acc);
int launch_fermion_kick(Ctx& c, const double* U64, const double* chi, const double* xi, double* p,
                        double eps, double* Fout, bool acc);
int launch_deriv_hop(Ctx& c, const double* U64, const double* v, const double* in, double* out,
                     bool dagger);
// Z1 = z1 - z1s (z1s may be NULL: Z1 = z1).
int launch_fg_assemble(Ctx& c, const double* U64, const double* chi, const double* xi,
                       const double* z1, const double* z1s, const double* z2, const double* v,
                       double* C, bool acc);
int launch_gauge_hvp(Ctx& c, const double* q, const double* v, double* C, bool acc);
int launch_axpy_links(Ctx& c, double* y, const double* x, double a, const double* z, double b);
int launch_drift(Ctx& c, double* q, const double* p, double eps);
// y = w + a x + b z on real link fields (w, z may be NULL).
// Spinors: y = w + a x.
int launch_spinor_lincomb(Ctx& c, double* y, const double* w, double a, const double* x);
int launch_lincomb(Ctx& c, double* y, const double* w, double a, const double* x, double b,
                   const double* z);
int launch_energies(Ctx& c, const double* q, const double* p, const double* phi, const double* xi,
                    double* K, double* SG, double* SF);
int launch_copy_links_masked(Ctx& c, double* dst, const double* src, const int* mask);

// Fused D^dag D (ddagd.cu).
int build_tile_table(sm_lattice* lat);
bool make_tile_tmaps(const sm_lattice* L, const float* in, const float* U, CUtensorMap* tin,
                     CUtensorMap* tU);
void big_tile_ranges(sm_lattice* lat);
// Chooses the strip height and each chain's block range of the streaming
// form (before the chain table is uploaded).
int stream_ranges(sm_lattice* lat);
int ddagd_stream_occupancy();
int cgt_fused_occupancy();
template <typename R>
int launch_ddagd(Ctx& c, const R* U, const R* in, R* out);

// Chain-resident CG (cg_chain.cu): one block per chain.
bool chain_cg_fits(const sm_lattice* L, int prec);
bool chain_variant_applies(const sm_lattice* L, int v);
bool big_chain_shape(const ChainInfo& ci);
constexpr int kChainVariants = SM_CG_VARIANTS;
// SM_MIXED kernels leave D x of the result in dx (FP64 [N][2][2]; the last
// FP64 reliable update computes it; zero where b = 0) when dx is not NULL,
// else use the workspace's scratch for it.
int chain_cg_launch(Ctx& c, const double* U64, const float* U32, const double* b, double* x,
                    const sm_cg_params& cg, double* dx = nullptr);

// Sets the launch attributes of the chain-resident kernel a solve with
// these parameters will use (done before a CUDA-graph capture).
int chain_cg_prepare(const sm_lattice* L, const sm_cg_params& cg);
// True if every solve with these parameters takes the chain-resident path.
bool chain_cg_selected(const sm_lattice* L, const sm_cg_params& cg);
int chain_cg_accumulate(Ctx& c);
// The kernel group of a chain of at most 4096 sites: 1-4 the column-pair
// kernels of 16 x 16, 32 x 32, 48 x 48 and 64 x 64 chains, 0 the strided
// kernel (any other shape).
int chain_group_kind(const sm::ChainInfo& ci);
int chain_cg_launch_list(Ctx& c, const double* U64, const float* U32, const double* b, double* x,
                         const sm_cg_params& cg, double* dx = nullptr);

// The tiled grid-wide mixed iteration (cg_tiled.cu) for batches of 2^18
// sites or more: n iterations of P, AP, XR on r, x, p (in place), Ap.
bool tiled_cg_applies(const sm_lattice* L);
int tiled_cg_iterate(Ctx& c, const float* U32, float* r, float* x, float* pa, float* pb,
                     float* Ap, double tol2, double delta2, int maxit, int n);
// Before a reliable update of the fused tiled form: x += alpha_x p for the
// chains about to be updated (their pending update of the iterate).
int tiled_cg_flush(Ctx& c, float* x, const float* pa, const float* pb,
                   const unsigned char* grid_mask);

// Kernel times of deferred solves and their site-iterations (solver.cu);
// call after the stream has been synchronised.
int profile_collect_deferred(const sm_lattice* L, const int* chain_iters);

// Blocks of the kernels that run after every chunk of CG iterations but
// work only when a reliable update is due (k_cg_res_d, k_cg_res_r,
// k_cgt_xflush): each loops over site blocks, so a chunk without an update
// costs a flag read per site block rather than a launch of every block.
inline unsigned res_grid(const sm_lattice* L) {
  return (unsigned)(L->nblocks < 2048 ? L->nblocks : 2048);
}

// CG on D^dag D (solver.cu).  b, x FP64; x is overwritten.  If iters/relres
// are non-NULL they receive host copies.  Synchronises (except in deferred
// mode).  If dx is not NULL, solves that compute D x of the result in FP64
// anyway (the chain-resident mixed ones, in their last reliable update) leave
// it there and set *have_dx; otherwise *have_dx is false and dx is untouched
// or scratch.
int cg_solve(Ctx& c, const double* U64, const float* U32, const double* b, double* x,
             const sm_cg_params& cg, int* iters, double* relres, double* dx = nullptr,
             bool* have_dx = nullptr);

}  // namespace sm
