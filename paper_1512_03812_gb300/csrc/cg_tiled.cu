// cg_tiled.cu -- the grid-wide mixed-precision CG iteration for large chains,
// built on the 64 x 16-tile fused D^dag D.
//
// One iteration is three launches over the chains still iterating:
//   P   p <- r + beta p                        (streaming, in place)
//   AP  A p = D^dag D p on tiles, with p^dag A p = |D p|^2 summed over each
//       tile's own sites and then over the chain's tiles -> alpha
//   XR  x <- x + alpha p, r <- r - alpha A p, |r|^2 -> beta, convergence
// The FP64 reliable updates, the state machine and the host loop are those of
// solver.cu; only the iteration body differs from its two-kernel form, whose
// stencil reads every neighbour through L1 and which stays in use for small
// batches.
#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "stream.cuh"
#include "tile.cuh"

namespace sm {

struct TiledArgs {
  Geo g;
  const int4* tiles;
  const int4* strips;  // streaming form (stream.cuh), if the lattice allows it
  int TT;
  const float* U;
  float* r;
  float* x;
  float* p;
  float* Ap;
  CgChain* cgc;
  double* partials;
  unsigned* counters;
  int* n_active;
  int* err;
  double tol2, delta2;
  int maxit;
};

__global__ void __launch_bounds__(kBlock) k_cgt_p(TiledArgs a) {
  const int c = a.g.blk_chain[blockIdx.x];
  const CgChain* cc = a.cgc + c;
  if (cc->state != 1) return;
  const ChainInfo ci = a.g.chains[c];
  const Site s = site_of(a.g, ci, c);
  if (!s.valid) return;
  const float beta = (float)cc->beta;
  st_sp(a.p, s.n, ld_sp_cg(a.r, s.n) + beta * ld_sp_cg(a.p, s.n));
}

// Sum over a block of kBT threads (16 warps); result in thread 0.
__device__ __forceinline__ double sum512(double v) {
  __shared__ double sh[kBT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < kBT / 32 ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

__global__ void __launch_bounds__(kBT) k_cgt_ap(TiledArgs a,
                                                const __grid_constant__ CUtensorMap tin,
                                                const __grid_constant__ CUtensorMap tU, int tma) {
  extern __shared__ __align__(128) float4 sm4[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ bool last;
  const int4 tile = a.tiles[blockIdx.x];
  const int c = tile.x;
  CgChain* cc = a.cgc + c;
  if (cc->state != 1) return;
  const ChainInfo ci = a.g.chains[c];
  float nrm = 0.f;
  ddagd_big_tile(sm4, ci, tile, a.U, a.p, a.Ap, &nrm, tma ? &tin : nullptr, tma ? &tU : nullptr,
                 &bar, a.err);
  // |D p|^2: block sum, then the chain's tiles in tile order (last block)
  const double part = sum512((double)nrm);
  if (threadIdx.x == 0) {
    __stcg(a.partials + blockIdx.x, part);
    __threadfence();
    last = atomicAdd(a.counters + c, 1u) == (unsigned)ci.ntb - 1u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tot = 0.0;
  for (int i = threadIdx.x; i < ci.ntb; i += kBT) tot += __ldcg(a.partials + ci.tb0 + i);
  tot = sum512(tot);
  if (threadIdx.x == 0) {
    a.counters[c] = 0u;
    if (tot > 0.0 && isfinite(tot)) {
      cc->alpha = cc->rr / tot;
    } else {
      cc->alpha = 0.0;
      cc->flags |= 2;
      cc->state = 0;
      atomicSub(a.n_active, 1);
    }
  }
}

// The same on the streaming form: one strip per warp, block partials in the
// chain's range of the strip table.
__global__ void __launch_bounds__(kSThreads, 4) k_cgt_ap_stream(TiledArgs a) {
  __shared__ __align__(16) float4 ring[kSWarps * kSRing];
  __shared__ double red[kSWarps];
  __shared__ bool last;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 s = a.strips[blockIdx.x * kSWarps + w];
  const int c = s.x;  // the same for every warp of the block
  CgChain* cc = a.cgc + c;
  if (cc->state != 1) return;
  const ChainInfo ci = a.g.chains[c];
  double v = ddagd_stream_strip<true>(ring + w * kSRing, a.g.chains, s, a.TT, a.U, a.p, a.Ap);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double part = 0.0;
#pragma unroll
    for (int k = 0; k < kSWarps; ++k) part += red[k];
    __stcg(a.partials + blockIdx.x, part);
    __threadfence();
    last = atomicAdd(a.counters + c, 1u) == (unsigned)ci.nsb - 1u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // |D p|^2 of the chain: its blocks' partials in block order
  double tot = 0.0;
  for (int i = threadIdx.x; i < ci.nsb; i += kSThreads) tot += __ldcg(a.partials + ci.sb0 + i);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
  __syncthreads();
  if (lane == 0) red[w] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    tot = 0.0;
#pragma unroll
    for (int k = 0; k < kSWarps; ++k) tot += red[k];
    a.counters[c] = 0u;
    if (tot > 0.0 && isfinite(tot)) {
      cc->alpha = cc->rr / tot;
    } else {
      cc->alpha = 0.0;
      cc->flags |= 2;
      cc->state = 0;
      atomicSub(a.n_active, 1);
    }
  }
}

int cgt_stream_occupancy() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cgt_ap_stream, kSThreads, 0) !=
      cudaSuccess)
    return 0;
  return n;
}

__global__ void __launch_bounds__(kBlock) k_cgt_xr(TiledArgs a) {
  const int c = a.g.blk_chain[blockIdx.x];
  CgChain* cc = a.cgc + c;
  if (cc->state != 1) return;
  const ChainInfo ci = a.g.chains[c];
  const Site s = site_of(a.g, ci, c);
  const float alpha = (float)cc->alpha;
  double v[1] = {0.0};
  if (s.valid) {
    st_sp(a.x, s.n, ld_sp_cg(a.x, s.n) + alpha * ld_sp_cg(a.p, s.n));
    const Sp<float> rv = ld_sp_cg(a.r, s.n) - alpha * ld_sp_cg(a.Ap, s.n);
    st_sp(a.r, s.n, rv);
    v[0] = (double)norm2(rv);
  }
  double tot[1];
  if (chain_reduce<1>(v, a.partials, a.counters, a.g, ci, c, tot) && threadIdx.x == 0) {
    const double rr = tot[0];
    cc->rr_prev = cc->rr;
    cc->rr = rr;
    cc->beta = rr / cc->rr_prev;
    cc->iters += 1;
    if (!isfinite(rr)) {
      cc->flags |= 2;
      cc->state = 0;
      atomicSub(a.n_active, 1);
    } else if (rr <= a.tol2 * cc->bb || cc->iters >= a.maxit) {
      cc->state = 2;  // wait for the FP64 check
      cc->need_update = 1;
    } else if (rr < a.delta2 * cc->rmax) {
      cc->need_update = 1;
    }
    cc->rmax = fmax(cc->rmax, rr);
  }
}

bool tiled_cg_applies(const sm_lattice* L) { return L->N >= (1 << 18); }

int tiled_cg_iterate(Ctx& c, const float* U32, float* r, float* x, float* p, float* Ap,
                     double tol2, double delta2, int maxit, int n) {
  TiledArgs a{};
  a.g = c.g;
  a.tiles = c.L->d_tiles_big;
  a.strips = c.L->d_stream;
  a.TT = c.L->stream_tt;
  a.U = U32;
  a.r = r;
  a.x = x;
  a.p = p;
  a.Ap = Ap;
  a.cgc = c.w.cgc;
  a.partials = c.w.partials;
  a.counters = c.w.counters;
  a.n_active = c.w.n_active;
  a.err = c.L->d_err;
  a.tol2 = tol2;
  a.delta2 = delta2;
  a.maxit = maxit;
  const bool stream = c.L->stream_ok;
  CUtensorMap tin, tU;
  int tma = 0;
  if (!stream) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_cgt_ap, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBigSmemBytes);
    if (e != cudaSuccess)
      return fail(SM_ERR_CUDA, "tiled CG attribute: %s", cudaGetErrorString(e));
    tma = make_tile_tmaps(c.L, p, U32, &tin, &tU) ? 1 : 0;
  }
  for (int k = 0; k < n; ++k) {
    k_cgt_p<<<c.grid(), kBlock, 0, c.s>>>(a);
    int rc = launched(c.st, "cgt_p");
    if (rc) return rc;
    if (stream)
      k_cgt_ap_stream<<<c.L->nstream, kSThreads, 0, c.s>>>(a);
    else
      k_cgt_ap<<<c.L->ntiles_big, kBT, kBigSmemBytes, c.s>>>(a, tin, tU, tma);
    if ((rc = launched(c.st, "cgt_ap"))) return rc;
    k_cgt_xr<<<c.grid(), kBlock, 0, c.s>>>(a);
    if ((rc = launched(c.st, "cgt_xr"))) return rc;
  }
  return SM_OK;
}

}  // namespace sm
