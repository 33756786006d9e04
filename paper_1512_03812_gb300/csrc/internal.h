// internal.h -- host-side declarations shared by the library's translation
// units: the lattice object, workspace carving, error reporting and the
// kernel launchers.
#pragma once

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
  int cg_variant;     // chain-resident mixed CG kernel chosen by sm_autotune_cg (-1: default)
  int device;
  int* h_pinned;  // small pinned host buffer for per-call readbacks
  cudaEvent_t ev[2];  // readback events of the CG loop
};

namespace sm {

// Sets the thread-local message and returns `code`.
int fail(int code, const char* fmt, ...);
// Counts one kernel launch and checks the launch for errors.
int launched(sm_stats* st, const char* what);

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
  int pad;
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
  // reductions
  double* partials;    // [4][nblocks]
  unsigned* counters;  // [nchains]
  CgChain* cgc;        // [nchains]
  double* out;         // [8][nchains]
  int* flags;          // [nchains] per-chain masks
  int* n_active;       // [1]
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

  int init(const sm_lattice* lat, void* ws, size_t nbytes, void* stream, sm_stats* stats);
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
int launch_fg_assemble(Ctx& c, const double* U64, const double* chi, const double* xi,
                       const double* z1, const double* z2, const double* v, double* C, bool acc);
int launch_gauge_hvp(Ctx& c, const double* q, const double* v, double* C, bool acc);
int launch_axpy_links(Ctx& c, double* y, const double* x, double a, const double* z, double b);
int launch_drift(Ctx& c, double* q, const double* p, double eps);
// y = w + a x + b z on real link fields (w, z may be NULL).
int launch_lincomb(Ctx& c, double* y, const double* w, double a, const double* x, double b,
                   const double* z);
int launch_energies(Ctx& c, const double* q, const double* p, const double* phi, const double* xi,
                    double* K, double* SG, double* SF);
int launch_copy_links_masked(Ctx& c, double* dst, const double* src, const int* mask);

// Fused D^dag D (ddagd.cu).
int build_tile_table(sm_lattice* lat);
template <typename R>
int launch_ddagd(Ctx& c, const R* U, const R* in, R* out);

// Chain-resident CG (cg_chain.cu): one block per chain.
bool chain_cg_fits(const sm_lattice* L, int prec);
bool chain_variant_applies(const sm_lattice* L, int v);
constexpr int kChainVariants = 4;
int chain_cg_launch(Ctx& c, const double* U64, const float* U32, const double* b, double* x,
                    const sm_cg_params& cg);

// CG on D^dag D (solver.cu).  b, x FP64; x is overwritten.  If iters/relres
// are non-NULL they receive host copies.  Synchronises.
int cg_solve(Ctx& c, const double* U64, const float* U32, const double* b, double* x,
             const sm_cg_params& cg, int* iters, double* relres);

}  // namespace sm
