// ddagd.cu -- fused D^dag D (Eq. fer_action) for lattices of any size.
//
// One thread block computes out = D^dag D in on a TX x TY tile of one chain.
// It stages `in` on the tile plus a 2-site halo and the links on the tile
// plus the sites the two stages touch, computes t = D in on the tile plus a
// 1-site ring into shared memory, and then D^dag t on the tile.  Global
// traffic is one read of `in` and U and one write of `out` per site (48 B in
// FP32, 96 B in FP64) instead of the 2x of two separate passes; the halo
// re-reads of neighbouring tiles are served by L2.  Coordinates wrap
// periodically per element, so tiles larger than a small lattice, partial
// edge tiles and ragged batches all work (the antiperiodic sign is in U).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "stream.cuh"
#include "tile.cuh"

namespace sm {

constexpr int kTX = 32, kTY = 8;             // tile, one site per thread in the D^dag stage
constexpr int kPX = kTX + 4, kPY = kTY + 4;  // `in` region: tile + 2-site halo
constexpr int kUX = kTX + 3, kUY = kTY + 3;  // links: x0-2 .. x0+TX, t0-2 .. t0+TY
constexpr int kDX = kTX + 2, kDY = kTY + 2;  // t = D in: tile + 1-site ring

template <typename R>
struct SpV;  // a spinor as stored in shared memory
template <>
struct SpV<float> {
  float4 v;
};
template <>
struct SpV<double> {
  double2 a, b;
};

__device__ __forceinline__ SpV<float> pack(Sp<float> s) {
  return {make_float4(s.a.re, s.a.im, s.b.re, s.b.im)};
}
__device__ __forceinline__ SpV<double> pack(Sp<double> s) {
  return {make_double2(s.a.re, s.a.im), make_double2(s.b.re, s.b.im)};
}
__device__ __forceinline__ Sp<float> unpack(const SpV<float>& s) {
  return {{s.v.x, s.v.y}, {s.v.z, s.v.w}};
}
__device__ __forceinline__ Sp<double> unpack(const SpV<double>& s) {
  return {{s.a.x, s.a.y}, {s.b.x, s.b.y}};
}

template <typename R>
__global__ void __launch_bounds__(kTX* kTY) k_ddagd_tile(const ChainInfo* __restrict__ chains,
                                                         const int4* __restrict__ tiles,
                                                         const R* __restrict__ U,
                                                         const R* __restrict__ in,
                                                         R* __restrict__ out) {
  __shared__ SpV<R> sp[kPY][kPX];
  __shared__ SpV<R> su[kUY][kUX];  // both links of a site, same storage as a spinor
  __shared__ SpV<R> st[kDY][kDX];
  const int4 tile = tiles[blockIdx.x];
  const ChainInfo ci = chains[tile.x];
  const int x0 = tile.y, t0 = tile.z, L = ci.L, T = ci.T;
  const long long off = ci.off;
  const int tid = threadIdx.x;

  // stage `in` and U, wrapping every coordinate periodically (tiles may be
  // larger than a small lattice)
  auto wx = [&](int x) { x = x < 0 ? x + L : x; while (x >= L) x -= L; return x; };
  auto wt = [&](int t) { t = t < 0 ? t + T : t; while (t >= T) t -= T; return t; };
  for (int i = tid; i < kPX * kPY; i += kTX * kTY) {
    const int ly = i / kPX, lx = i - ly * kPX;
    const long long n = off + wx(x0 - 2 + lx) + (long long)L * wt(t0 - 2 + ly);
    sp[ly][lx] = pack(ld_sp(in, n));
  }
  for (int i = tid; i < kUX * kUY; i += kTX * kTY) {
    const int ly = i / kUX, lx = i - ly * kUX;
    const long long n = off + wx(x0 - 2 + lx) + (long long)L * wt(t0 - 2 + ly);
    const Lk<R> u = ld_lk(U, n);
    su[ly][lx] = pack(Sp<R>{u.x, u.t});
  }
  __syncthreads();

  // t = D in on the tile plus a 1-site ring: ring site (dx, dy) is lattice
  // site (x0 - 1 + dx, t0 - 1 + dy), i.e. sp[dy + 1][dx + 1], su[dy + 1][dx + 1]
  const R diag = (R)(2.0 + ci.m0);
  for (int i = tid; i < kDX * kDY; i += kTX * kTY) {
    const int dy = i / kDX, dx = i - dy * kDX;
    const int px = dx + 1, py = dy + 1;
    // the halo of the staged region (checked in the debug build)
    const int pxp = (int)SM_IDX(px + 1, kPX, 20), pxm = (int)SM_IDX(px - 1, kPX, 21);
    const int pyp = (int)SM_IDX(py + 1, kPY, 22), pym = (int)SM_IDX(py - 1, kPY, 23);
    const Sp<R> u = unpack(su[(int)SM_IDX(py, kUY, 24)][(int)SM_IDX(px, kUX, 25)]);
    const Sp<R> o = hop_sum<false, R>(unpack(sp[py][pxp]), unpack(sp[py][pxm]),
                                      unpack(sp[pyp][px]), unpack(sp[pym][px]), u.a,
                                      unpack(su[py][pxm]).a, u.b, unpack(su[pym][px]).b);
    st[dy][dx] = pack(diag * unpack(sp[py][px]) - (R)0.5 * o);
  }
  __syncthreads();

  // out = D^dag t on the tile
  const int ty = tid / kTX, tx = tid - ty * kTX;
  const int x = x0 + tx, t = t0 + ty;
  if (x >= L || t >= T) return;
  const int dx = tx + 1, dy = ty + 1;  // in st
  const int ux = (int)SM_IDX(tx + 2, kUX, 26), uy = (int)SM_IDX(ty + 2, kUY, 27);  // in su
  const int dxp = (int)SM_IDX(dx + 1, kDX, 28), dyp = (int)SM_IDX(dy + 1, kDY, 29);
  const Sp<R> u = unpack(su[uy][ux]);
  const Sp<R> o = hop_sum<true, R>(unpack(st[dy][dxp]), unpack(st[dy][dx - 1]),
                                   unpack(st[dyp][dx]), unpack(st[dy - 1][dx]), u.a,
                                   unpack(su[uy][ux - 1]).a, u.b, unpack(su[uy - 1][ux]).b);
  st_sp(out, off + x + (long long)L * t, diag * unpack(st[dy][dx]) - (R)0.5 * o);
}

__global__ void __launch_bounds__(kBT) k_ddagd_tile_big(const ChainInfo* __restrict__ chains,
                                                        const int4* __restrict__ tiles,
                                                        const float* __restrict__ U,
                                                        const float* __restrict__ in,
                                                        float* __restrict__ out,
                                                        const __grid_constant__ CUtensorMap tin,
                                                        const __grid_constant__ CUtensorMap tU,
                                                        int tma, int* err, int spin) {
  extern __shared__ __align__(128) float4 sm4[];
  __shared__ __align__(8) unsigned long long bar;
  const int4 tile = tiles[blockIdx.x];
  ddagd_big_tile(sm4, chains[tile.x], tile, U, in, out, nullptr, tma ? &tin : nullptr,
                 tma ? &tU : nullptr, &bar, err, spin);
}

// Streaming form: one strip per warp (stream.cuh).
__global__ void __launch_bounds__(kSThreads, 4) k_ddagd_stream(const ChainInfo* __restrict__ chains,
                                                             const int4* __restrict__ strips,
                                                             int TT, const float* __restrict__ U,
                                                             const float* __restrict__ in,
                                                             float* __restrict__ out) {
  __shared__ __align__(16) float4 ring[kSWarps * kSRing];
  const int w = threadIdx.x >> 5;
  ddagd_stream_strip<false>(ring + w * kSRing, chains, strips[blockIdx.x * kSWarps + w], TT, U,
                            in, out);
}

int ddagd_stream_occupancy() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ddagd_stream, kSThreads, 0) !=
      cudaSuccess)
    return 0;
  return n;
}

// Strips per chain for strip height TT, and the blocks they fill.
static long long stream_blocks(const sm_lattice* lat, int TT) {
  long long nb = 0;
  for (const ChainInfo& ci : lat->chains) {
    const long long strips =
        (long long)((ci.L + kSOut - 1) / kSOut) * ((ci.T + TT - 1) / TT);
    nb += (strips + kSWarps - 1) / kSWarps;
  }
  return nb;
}

// The lowest strip height whose blocks all fit on the GPU at once (one wave)
// for a kernel that holds `occ` blocks per SM; launches with fewer strips per
// SM than that lose bandwidth.
static int stream_height(const sm_lattice* lat, int nsm, int occ) {
  const long long slots = (long long)nsm * occ;
  int tmax = 0;
  for (const ChainInfo& ci : lat->chains) tmax = std::max(tmax, ci.T);
  int lo = 8, hi = std::max(8, tmax);
  if (stream_blocks(lat, hi) > slots) return 32;  // more than one wave whatever the height
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (stream_blocks(lat, mid) <= slots) hi = mid; else lo = mid + 1;
  }
  return lo;
}

int stream_ranges(sm_lattice* lat) {
  // every chain must be wide enough that the 64-column windows waste little
  // (at most 30 % more columns than the lattice has)
  lat->stream_ok = lat->N >= (1 << 18);
  for (const ChainInfo& ci : lat->chains)
    if (10LL * kSW * ((ci.L + kSOut - 1) / kSOut) > 13LL * ci.L) lat->stream_ok = false;
  if (!lat->stream_ok) return SM_OK;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(SM_ERR_CUDA, "device attribute");
  const int occ_d = ddagd_stream_occupancy(), occ_cg = cgt_fused_occupancy();
  if (occ_d <= 0 || occ_cg <= 0) return fail(SM_ERR_CUDA, "streaming D^dag D: no occupancy");
  // the D^dag D and the CG iteration keep their own strip tables: the CG
  // kernel holds fewer blocks per SM (more registers, a larger ring)
  lat->stream_tt = stream_height(lat, nsm, occ_d);
  lat->nstream = (int)stream_blocks(lat, lat->stream_tt);
  lat->stream_tt_cg = stream_height(lat, nsm, occ_cg);
  int first = 0;
  for (ChainInfo& ci : lat->chains) {
    const long long strips = (long long)((ci.L + kSOut - 1) / kSOut) *
                             ((ci.T + lat->stream_tt_cg - 1) / lat->stream_tt_cg);
    ci.sb0 = first;
    ci.nsb = (int)((strips + kSWarps - 1) / kSWarps);
    first += ci.nsb;
  }
  lat->nstream_cg = first;
  return SM_OK;
}

// {chain, xs, ts, dir} per warp, kSWarps per block and a chain's last block
// padded with {chain, 0, 0, 0}; vertically adjacent strips walk in opposite
// directions
static int make_strips(const sm_lattice* lat, int TT, int4** d) {
  std::vector<int4> t;
  for (int c = 0; c < lat->nchains; ++c) {
    const ChainInfo& ci = lat->chains[c];
    const size_t first = t.size();
    for (int y = 0, k = 0; y < ci.T; y += TT, ++k)
      for (int x = 0; x < ci.L; x += kSOut) t.push_back(make_int4(c, x, y, 1 + (k & 1)));
    while ((t.size() - first) % kSWarps) t.push_back(make_int4(c, 0, 0, 0));
  }
  cudaError_t e = cudaMalloc(d, sizeof(int4) * t.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(*d, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "strip table: %s", cudaGetErrorString(e));
  return SM_OK;
}

// Candidate strip heights of the streaming D^dag D for this lattice: the
// lowest heights whose blocks fit on the GPU in 1, 2, 3 and 4 waves, and two
// and four times the one-wave height (taller strips: fewer halo re-reads,
// fewer blocks), at most the tallest chain, each once, ascending.
static std::vector<int> stream_candidates(const sm_lattice* lat, int nsm, int occ) {
  int tmax = 0;
  for (const ChainInfo& ci : lat->chains) tmax = std::max(tmax, ci.T);
  std::vector<int> c;
  for (int w = 1; w <= 4; ++w) c.push_back(stream_height(lat, nsm, occ * w));
  const int t1 = c[0];
  c.push_back(2 * t1);
  c.push_back(4 * t1);
  for (int& v : c) v = std::max(8, std::min(v, std::max(8, tmax)));
  std::sort(c.begin(), c.end());
  c.erase(std::unique(c.begin(), c.end()), c.end());
  return c;
}

static int build_stream_table(sm_lattice* lat) {
  if (!lat->stream_ok) return SM_OK;
  const int rc = make_strips(lat, lat->stream_tt, &lat->d_stream);
  if (rc) return rc;
  return make_strips(lat, lat->stream_tt_cg, &lat->d_stream_cg);
}

// Tensor maps of `in` and U for TMA staging (single-chain lattices large
// enough for interior tiles).  Returns false where TMA is not used.
bool make_tile_tmaps(const sm_lattice* L, const float* in, const float* U, CUtensorMap* tin,
                     CUtensorMap* tU) {
  if (L->nchains != 1) return false;
  const ChainInfo& ci = L->chains[0];
  if (ci.L < kBX + 4 || ci.T < kBY + 4) return false;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  if (!encode) return false;
  const cuuint64_t dims[2] = {2 * (cuuint64_t)ci.L, (cuuint64_t)ci.T};
  const cuuint64_t strides[1] = {16 * (cuuint64_t)ci.L};
  const cuuint32_t ebox[2] = {1, 1};
  const cuuint32_t bin[2] = {2 * kBPX, kBPY}, bU[2] = {2 * kBUX, kBUY};
  auto enc = [&](CUtensorMap* m, const float* base, const cuuint32_t* box) {
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<float*>(base), dims, strides,
                  box, ebox, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
  };
  return enc(tin, in, bin) && enc(tU, U, bU);
}

static int make_tiles(sm_lattice* lat, int tx, int ty, int4** d, int* n) {
  std::vector<int4> t;
  for (int c = 0; c < lat->nchains; ++c) {
    const ChainInfo& ci = lat->chains[c];
    for (int y = 0; y < ci.T; y += ty)
      for (int x = 0; x < ci.L; x += tx) t.push_back(make_int4(c, x, y, 0));
  }
  cudaError_t e = cudaMalloc(d, sizeof(int4) * t.size());
  if (e == cudaSuccess) e = cudaMemcpy(*d, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "tile table: %s", cudaGetErrorString(e));
  *n = (int)t.size();
  return SM_OK;
}

// Each chain's range in the 64 x 16 tile table (before the chain table is
// uploaded).
void big_tile_ranges(sm_lattice* lat) {
  int first = 0;
  for (ChainInfo& ci : lat->chains) {
    ci.tb0 = first;
    ci.ntb = ((ci.L + kBX - 1) / kBX) * ((ci.T + kBY - 1) / kBY);
    first += ci.ntb;
  }
}

// Tile table of a lattice: {chain, x0, t0, 0} per tile (at lattice creation).
int build_tile_table(sm_lattice* lat) {
  int rc = make_tiles(lat, kTX, kTY, &lat->d_tiles, &lat->ntiles);
  if (rc) return rc;
  if ((rc = make_tiles(lat, kBX, kBY, &lat->d_tiles_big, &lat->ntiles_big))) return rc;
  return build_stream_table(lat);
}

template <typename R>
int launch_ddagd(Ctx& c, const R* U, const R* in, R* out) {
  if (sizeof(R) == 4 && c.L->stream_ok) {
    k_ddagd_stream<<<c.L->nstream, kSThreads, 0, c.s>>>(c.L->d_chains, c.L->d_stream,
                                                         c.L->stream_tt, (const float*)U,
                                                         (const float*)in, (float*)out);
    return launched(c.st, "ddagd_stream");
  }
  if (sizeof(R) == 4 && c.L->N >= (1 << 18)) {
    // large FP32 batches of narrow chains: big tiles (the small-tile table
    // stays for small batches)
    const size_t smem = kBigSmemBytes;
    cudaError_t e = cudaFuncSetAttribute(k_ddagd_tile_big,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(SM_ERR_CUDA, "ddagd attribute: %s", cudaGetErrorString(e));
    CUtensorMap tin, tU;
    const bool tma = make_tile_tmaps(c.L, (const float*)in, (const float*)U, &tin, &tU);
    k_ddagd_tile_big<<<c.L->ntiles_big, kBT, smem, c.s>>>(
        c.L->d_chains, c.L->d_tiles_big, (const float*)U, (const float*)in, (float*)out, tin, tU,
        tma ? 1 : 0, c.L->d_err, c.L->tma_spin);
    return launched(c.st, "ddagd_tile_big");
  }
  k_ddagd_tile<R><<<c.L->ntiles, kTX * kTY, 0, c.s>>>(c.L->d_chains, c.L->d_tiles, U, in, out);
  return launched(c.st, "ddagd_tile");
}
template int launch_ddagd<float>(Ctx&, const float*, const float*, float*);
template int launch_ddagd<double>(Ctx&, const double*, const double*, double*);

}  // namespace sm

using namespace sm;

extern "C" int sm_autotune_ddagd(sm_lattice* lat, const float* U32, const float* in, float* out,
                                 int* height, int* heights, double* ms, void* stream) {
  if (!lat || !U32 || !in || !out) return fail(SM_ERR_ARG, "sm_autotune_ddagd: NULL argument");
  if ((((uintptr_t)U32) | ((uintptr_t)in) | ((uintptr_t)out)) & 15)
    return fail(SM_ERR_ARG, "sm_autotune_ddagd: unaligned field");
  if (in == out) return fail(SM_ERR_ARG, "sm_autotune_ddagd: in and out alias");
  if (heights)
    for (int k = 0; k < SM_DDAGD_HEIGHTS; ++k) heights[k] = -1;
  if (ms)
    for (int k = 0; k < SM_DDAGD_HEIGHTS; ++k) ms[k] = -1.0;
  if (!lat->stream_ok) {
    if (height) *height = 0;  // the tiled forms serve this lattice: nothing to tune
    return SM_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int nsm = 0;
  cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, lat->device);
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "sm_autotune_ddagd: %s", cudaGetErrorString(e));
  const std::vector<int> cand = stream_candidates(lat, nsm, ddagd_stream_occupancy());
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "sm_autotune_ddagd: %s", cudaGetErrorString(e));
  const int reps = 10;
  int best = lat->stream_tt;
  float best_ms = -1.f;
  int rc = SM_OK;
  for (size_t k = 0; k < cand.size() && k < (size_t)SM_DDAGD_HEIGHTS && rc == SM_OK; ++k) {
    const int TT = cand[k];
    int4* table = nullptr;
    if ((rc = make_strips(lat, TT, &table))) break;
    const unsigned nb = (unsigned)stream_blocks(lat, TT);
    for (int r = 0; r < 2; ++r)  // warm-up
      k_ddagd_stream<<<nb, kSThreads, 0, s>>>(lat->d_chains, table, TT, U32, in, out);
    e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r)
      k_ddagd_stream<<<nb, kSThreads, 0, s>>>(lat->d_chains, table, TT, U32, in, out);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaFree(table);
    if (e != cudaSuccess) {
      rc = fail(SM_ERR_CUDA, "sm_autotune_ddagd: %s", cudaGetErrorString(e));
      break;
    }
    add_launches(reps + 2);
    t /= reps;
    if (heights) heights[k] = TT;
    if (ms) ms[k] = t;
    if (best_ms < 0.f || t < best_ms) {
      best_ms = t;
      best = TT;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (best != lat->stream_tt) {
    int4* table = nullptr;
    if ((rc = make_strips(lat, best, &table))) return rc;
    cudaFree(lat->d_stream);
    lat->d_stream = table;
    lat->stream_tt = best;
    lat->nstream = (int)stream_blocks(lat, best);
  }
  if (height) *height = lat->stream_tt;
  return SM_OK;
}
