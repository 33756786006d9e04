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

#include <vector>

#include "common.cuh"
#include "internal.h"
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
    const Sp<R> u = unpack(su[py][px]);
    const Sp<R> o = hop_sum<false, R>(unpack(sp[py][px + 1]), unpack(sp[py][px - 1]),
                                      unpack(sp[py + 1][px]), unpack(sp[py - 1][px]), u.a,
                                      unpack(su[py][px - 1]).a, u.b, unpack(su[py - 1][px]).b);
    st[dy][dx] = pack(diag * unpack(sp[py][px]) - (R)0.5 * o);
  }
  __syncthreads();

  // out = D^dag t on the tile
  const int ty = tid / kTX, tx = tid - ty * kTX;
  const int x = x0 + tx, t = t0 + ty;
  if (x >= L || t >= T) return;
  const int dx = tx + 1, dy = ty + 1;  // in st
  const int ux = tx + 2, uy = ty + 2;  // in su
  const Sp<R> u = unpack(su[uy][ux]);
  const Sp<R> o = hop_sum<true, R>(unpack(st[dy][dx + 1]), unpack(st[dy][dx - 1]),
                                   unpack(st[dy + 1][dx]), unpack(st[dy - 1][dx]), u.a,
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
                                                        int tma, int* err) {
  extern __shared__ __align__(128) float4 sm4[];
  __shared__ __align__(8) unsigned long long bar;
  const int4 tile = tiles[blockIdx.x];
  ddagd_big_tile(sm4, chains[tile.x], tile, U, in, out, nullptr, tma ? &tin : nullptr,
                 tma ? &tU : nullptr, &bar, err);
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
  const int rc = make_tiles(lat, kTX, kTY, &lat->d_tiles, &lat->ntiles);
  if (rc) return rc;
  return make_tiles(lat, kBX, kBY, &lat->d_tiles_big, &lat->ntiles_big);
}

template <typename R>
int launch_ddagd(Ctx& c, const R* U, const R* in, R* out) {
  if (sizeof(R) == 4 && c.L->N >= (1 << 18)) {
    // large FP32 batches: big tiles (the small-tile table stays for small ones)
    const size_t smem = kBigSmemBytes;
    cudaError_t e = cudaFuncSetAttribute(k_ddagd_tile_big,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(SM_ERR_CUDA, "ddagd attribute: %s", cudaGetErrorString(e));
    CUtensorMap tin, tU;
    const bool tma = make_tile_tmaps(c.L, (const float*)in, (const float*)U, &tin, &tU);
    k_ddagd_tile_big<<<c.L->ntiles_big, kBT, smem, c.s>>>(
        c.L->d_chains, c.L->d_tiles_big, (const float*)U, (const float*)in, (float*)out, tin, tU,
        tma ? 1 : 0, c.L->d_err);
    return launched(c.st, "ddagd_tile_big");
  }
  k_ddagd_tile<R><<<c.L->ntiles, kTX * kTY, 0, c.s>>>(c.L->d_chains, c.L->d_tiles, U, in, out);
  return launched(c.st, "ddagd_tile");
}
template int launch_ddagd<float>(Ctx&, const float*, const float*, float*);
template int launch_ddagd<double>(Ctx&, const double*, const double*, double*);

}  // namespace sm
