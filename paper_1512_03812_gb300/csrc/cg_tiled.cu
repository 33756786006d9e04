// cg_tiled.cu -- the grid-wide mixed-precision CG iteration for large
// batches (2^18 sites or more).
//
// Batches whose chains all take the streaming D^dag D (stream.cuh) iterate
// with two launches (the fused form below): F forms p = r + beta p_old on
// every strip window, stores p and advances x at the strip's own sites, and
// computes A p = D^dag D p with |D p|^2 -> alpha; R updates r and |r|^2 ->
// beta.  Other large batches iterate with three launches on 64 x 16 tiles:
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
  float* p;   // the tiled (non-streaming) form: p in place
  float* pb;  // the fused streaming form: p double-buffered (p, pb), CgChain::par
  float* Ap;
  CgChain* cgc;
  double* partials;
  unsigned* counters;
  int* n_active;  // [0] chains still iterating, [1] chains due a reliable update
  int* err;
  int spin;  // polls of the first TMA wait
  const unsigned char* grid_mask;  // hybrid solves: 0 for chains solved chain-resident
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
                 &bar, a.err, a.spin);
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

// The fused streaming iteration (batches whose chains all take the
// streaming D^dag D).  Kernel F: p = r + beta p_old on every strip window,
// p stored at the strip's own sites, x += alpha_x p_old there (the previous
// iteration's update of the iterate), A p = D^dag D p, |D p|^2 -> alpha; the
// chain's p buffers swap.  Kernel R: r -= alpha A p, |r|^2 -> beta, and
// alpha_x = alpha for the next F.  Per site and iteration: r, p_old, U read
// and p, A p written by F, x advanced in L2, r and A p read and r written by
// R: 160 bytes instead of the 192 of P, AP, XR.
__global__ void __launch_bounds__(kSThreads, 3) k_cgt_f(TiledArgs a) {
  extern __shared__ __align__(16) float4 ringf[];
  __shared__ double red[kSWarps];
  __shared__ bool last;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 s = a.strips[blockIdx.x * kSWarps + w];
  const int c = s.x;  // the same for every warp of the block
  CgChain* cc = a.cgc + c;
  if (cc->state != 1) return;
  const ChainInfo ci = a.g.chains[c];
  const int par = cc->par;
  CgFuse f;
  f.pold = par ? a.pb : a.p;
  f.pnew = par ? a.p : a.pb;
  f.x = a.x;
  f.beta = (float)cc->beta;
  f.alpha_x = (float)cc->alpha_x;
  double v = ddagd_stream_strip_cg(ringf + w * kSRingCG, a.g.chains, s, a.TT, a.U, a.r, a.Ap, f);
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
    cc->par = par ^ 1;  // p is now in the other buffer
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

// Kernel R on the same strips as F (one strip per warp, a chain's blocks
// reduced in block order by its last block): every lane streams the rows of
// its strip, two columns at a time, with several rows' loads in flight.
__global__ void __launch_bounds__(kSThreads) k_cgt_r(TiledArgs a) {
  __shared__ double red[kSWarps];
  __shared__ bool last;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 s = a.strips[blockIdx.x * kSWarps + w];
  const int c = s.x;
  CgChain* cc = a.cgc + c;
  if (cc->state != 1) return;
  const ChainInfo ci = a.g.chains[c];
  const float alpha = (float)cc->alpha;
  double v = 0.0;
  if (s.w) {
    const int L = ci.L, ncols = min(kSOut, L - s.y), nr = min(a.TT, ci.T - s.z);
    const bool c0 = lane < ncols, c1 = lane + 32 < ncols;
    float4* r4 = reinterpret_cast<float4*>(a.r) + ci.off + s.y + (long long)L * s.z;
    const float4* ap4 = reinterpret_cast<const float4*>(a.Ap) + ci.off + s.y + (long long)L * s.z;
    float acc = 0.f;
    // four rows at a time: all their loads are issued before any store (the
    // compiler cannot move a load of r above a store to r by itself)
    constexpr int G = 4;
    for (int t0 = 0; t0 < nr; t0 += G) {
      float4 rl[G][2], al[G][2];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const long long o = (long long)L * (t0 + g) + lane;
        const bool in_rows = t0 + g < nr;
        if (in_rows && c0) {
          rl[g][0] = __ldcg(r4 + o);
          al[g][0] = __ldcg(ap4 + o);
        }
        if (in_rows && c1) {
          rl[g][1] = __ldcg(r4 + o + 32);
          al[g][1] = __ldcg(ap4 + o + 32);
        }
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const long long o = (long long)L * (t0 + g) + lane;
        const bool in_rows = t0 + g < nr;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (in_rows && (k ? c1 : c0)) {
            const Sp<float> rv = f4sp(rl[g][k]) - alpha * f4sp(al[g][k]);
            __stcg(r4 + o + 32 * k, make_float4(rv.a.re, rv.a.im, rv.b.re, rv.b.im));
            acc += norm2(rv);
          }
        }
      }
    }
    v = (double)acc;
  }
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
  double tot = 0.0;
  for (int i = threadIdx.x; i < ci.nsb; i += kSThreads) tot += __ldcg(a.partials + ci.sb0 + i);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
  __syncthreads();
  if (lane == 0) red[w] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    double rr = 0.0;
#pragma unroll
    for (int k = 0; k < kSWarps; ++k) rr += red[k];
    a.counters[c] = 0u;
    cc->alpha_x = cc->alpha;
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
      mark_update(cc, a.n_active + 1);
    } else if (rr < a.delta2 * cc->rmax) {
      mark_update(cc, a.n_active + 1);
    }
    cc->rmax = fmax(cc->rmax, rr);
  }
}

// x += alpha_x p for the chains about to take a reliable update (a block
// visits the site blocks blockIdx.x, + gridDim.x, ...)
__global__ void __launch_bounds__(kBlock) k_cgt_xflush(TiledArgs a) {
  if (a.n_active[1] == 0) return;  // no chain is due an update
  for (int blk = blockIdx.x; blk < a.g.nblocks; blk += gridDim.x) {
    const int c = a.g.blk_chain[blk];
    if (a.grid_mask && !a.grid_mask[c]) continue;
    const CgChain* cc = a.cgc + c;
    if (!cc->need_update || cc->alpha_x == 0.0) continue;
    const ChainInfo ci = a.g.chains[c];
    const Site s = site_of(a.g, ci, c, blk);
    if (!s.valid) continue;
    const float* p = cc->par ? a.pb : a.p;
    st_sp(a.x, s.n, ld_sp_cg(a.x, s.n) + (float)cc->alpha_x * ld_sp_cg(p, s.n));
  }
}

int cgt_fused_occupancy() {
  int n = 0;
  if (cudaFuncSetAttribute(k_cgt_f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(float4) * kSWarps * kSRingCG)) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cgt_f, kSThreads,
                                                    sizeof(float4) * kSWarps * kSRingCG) !=
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
      mark_update(cc, a.n_active + 1);
    } else if (rr < a.delta2 * cc->rmax) {
      mark_update(cc, a.n_active + 1);
    }
    cc->rmax = fmax(cc->rmax, rr);
  }
}

bool tiled_cg_applies(const sm_lattice* L) { return L->N >= (1 << 18); }

int tiled_cg_flush(Ctx& c, float* x, const float* pa, const float* pb,
                   const unsigned char* grid_mask) {
  TiledArgs a{};
  a.g = c.g;
  a.grid_mask = grid_mask;
  a.x = x;
  a.p = const_cast<float*>(pa);
  a.pb = const_cast<float*>(pb);
  a.cgc = c.w.cgc;
  a.n_active = c.w.n_active;
  k_cgt_xflush<<<dim3(res_grid(c.L)), kBlock, 0, c.s>>>(a);
  return launched(c.st, "cgt_xflush");
}

int tiled_cg_iterate(Ctx& c, const float* U32, float* r, float* x, float* p, float* pb,
                     float* Ap, double tol2, double delta2, int maxit, int n) {
  TiledArgs a{};
  a.g = c.g;
  a.tiles = c.L->d_tiles_big;
  a.strips = c.L->d_stream_cg;
  a.TT = c.L->stream_tt_cg;
  a.U = U32;
  a.r = r;
  a.x = x;
  a.p = p;
  a.pb = pb;
  a.Ap = Ap;
  a.cgc = c.w.cgc;
  a.partials = c.w.partials;
  a.counters = c.w.counters;
  a.n_active = c.w.n_active;
  a.err = c.L->d_err;
  a.spin = c.L->tma_spin;
  a.tol2 = tol2;
  a.delta2 = delta2;
  a.maxit = maxit;
  const bool stream = c.L->stream_ok;
  if (stream) {
    const size_t smem = sizeof(float4) * kSWarps * kSRingCG;
    const cudaError_t e =
        cudaFuncSetAttribute(k_cgt_f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
      return fail(SM_ERR_CUDA, "fused CG attribute: %s", cudaGetErrorString(e));
    for (int k = 0; k < n; ++k) {
      k_cgt_f<<<c.L->nstream_cg, kSThreads, smem, c.s>>>(a);
      int rc = launched(c.st, "cgt_f");
      if (rc) return rc;
      k_cgt_r<<<c.L->nstream_cg, kSThreads, 0, c.s>>>(a);
      if ((rc = launched(c.st, "cgt_r"))) return rc;
    }
    return SM_OK;
  }
  const cudaError_t e =
      cudaFuncSetAttribute(k_cgt_ap, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBigSmemBytes);
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "tiled CG attribute: %s", cudaGetErrorString(e));
  CUtensorMap tin, tU;
  const int tma = make_tile_tmaps(c.L, p, U32, &tin, &tU) ? 1 : 0;
  for (int k = 0; k < n; ++k) {
    k_cgt_p<<<c.grid(), kBlock, 0, c.s>>>(a);
    int rc = launched(c.st, "cgt_p");
    if (rc) return rc;
    k_cgt_ap<<<c.L->ntiles_big, kBT, kBigSmemBytes, c.s>>>(a, tin, tU, tma);
    if ((rc = launched(c.st, "cgt_ap"))) return rc;
    k_cgt_xr<<<c.grid(), kBlock, 0, c.s>>>(a);
    if ((rc = launched(c.st, "cgt_xr"))) return rc;
  }
  return SM_OK;
}

}  // namespace sm
