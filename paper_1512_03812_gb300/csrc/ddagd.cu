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
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"
#include "internal.h"

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

// FP32 form for large lattices: 64 x 16 tiles (4 output sites per thread,
// halo overhead 1.33x on `in` instead of 1.69x), staged with cp.async:
// every thread issues all of its 16-byte global -> shared copies before one
// wait, so a block has its whole 42 KB region in flight.  Interior tiles
// (whose region needs no periodic wrap) skip the wrap arithmetic.
constexpr int kBX = 64, kBY = 16, kBT = 512;
constexpr int kBPX = kBX + 4, kBPY = kBY + 4;
constexpr int kBUX = kBX + 3, kBUY = kBY + 3;
constexpr int kBDX = kBX + 2, kBDY = kBY + 2;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__global__ void __launch_bounds__(kBT) k_ddagd_tile_big(const ChainInfo* __restrict__ chains,
                                                        const int4* __restrict__ tiles,
                                                        const float* __restrict__ U,
                                                        const float* __restrict__ in,
                                                        float* __restrict__ out) {
  extern __shared__ float4 sm4[];
  float4* sp = sm4;                   // [kBPY][kBPX]
  float4* su = sp + kBPX * kBPY;      // [kBUY][kBUX]
  float4* st = su + kBUX * kBUY;      // [kBDY][kBDX]
  const int4 tile = tiles[blockIdx.x];
  const ChainInfo ci = chains[tile.x];
  const int x0 = tile.y, t0 = tile.z, L = ci.L, T = ci.T;
  const long long off = ci.off;
  const int tid = threadIdx.x;
  const float4* in4 = reinterpret_cast<const float4*>(in) + off;
  const float4* U4 = reinterpret_cast<const float4*>(U) + off;
  const bool interior = x0 >= 2 && x0 + kBX + 2 <= L && t0 >= 2 && t0 + kBY + 2 <= T;
  if (interior) {
    const float4* pin = in4 + (x0 - 2) + (long long)L * (t0 - 2);
    const float4* pU = U4 + (x0 - 2) + (long long)L * (t0 - 2);
    for (int i = tid; i < kBPX * kBPY; i += kBT) {
      const int ly = i / kBPX, lx = i - ly * kBPX;
      cp_async16(sp + i, pin + lx + (long long)L * ly);
    }
    for (int i = tid; i < kBUX * kBUY; i += kBT) {
      const int ly = i / kBUX, lx = i - ly * kBUX;
      cp_async16(su + i, pU + lx + (long long)L * ly);
    }
  } else {
    auto wx = [&](int x) { x %= L; return x < 0 ? x + L : x; };
    auto wt = [&](int t) { t %= T; return t < 0 ? t + T : t; };
    for (int i = tid; i < kBPX * kBPY; i += kBT) {
      const int ly = i / kBPX, lx = i - ly * kBPX;
      cp_async16(sp + i, in4 + wx(x0 - 2 + lx) + (long long)L * wt(t0 - 2 + ly));
    }
    for (int i = tid; i < kBUX * kBUY; i += kBT) {
      const int ly = i / kBUX, lx = i - ly * kBUX;
      cp_async16(su + i, U4 + wx(x0 - 2 + lx) + (long long)L * wt(t0 - 2 + ly));
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();

  const float diag = (float)(2.0 + ci.m0);
  auto S = [](float4 v) { return Sp<float>{{v.x, v.y}, {v.z, v.w}}; };
  // the link of the x (t) direction of a site: one 8-byte half of its float4
  const float2* su2 = reinterpret_cast<const float2*>(su);
  auto UX = [&](int u) { const float2 v = su2[2 * u]; return Cx<float>{v.x, v.y}; };
  auto UT = [&](int u) { const float2 v = su2[2 * u + 1]; return Cx<float>{v.x, v.y}; };
  // t = D in on the (kBX + 2) x (kBY + 2) region.  Threads 0 .. 383 walk the
  // 64 main columns in 6 strips of 3 rows (warps stay on one row: no bank
  // conflicts; t-neighbours and U_t(n - t) come from registers); threads
  // 384 .. 419 do the two halo columns site by site.
  constexpr int kDRows = kBDY / 6;
  auto dsite = [&](int dx, int dy, const Sp<float>& pm, const Sp<float>& pc,
                   const Sp<float>& pn, Cx<float> utm) {
    const int p = (dy + 1) * kBPX + dx + 1, u = (dy + 1) * kBUX + dx + 1;
    const float4 uu = su[u];
    const Sp<float> o = hop_sum<false, float>(S(sp[p + 1]), S(sp[p - 1]), pn, pm, {uu.x, uu.y},
                                              UX(u - 1), {uu.z, uu.w}, utm);
    const Sp<float> tv = diag * pc - 0.5f * o;
    st[dy * kBDX + dx] = make_float4(tv.a.re, tv.a.im, tv.b.re, tv.b.im);
    return Cx<float>{uu.z, uu.w};
  };
  if (tid < 6 * kBX) {
    const int dx = tid % kBX + 1, dy0 = (tid / kBX) * kDRows;
    int p = (dy0 + 1) * kBPX + dx + 1;
    Sp<float> pm = S(sp[p - kBPX]), pc = S(sp[p]);
    Cx<float> utm = UT((dy0 + 1) * kBUX + dx + 1 - kBUX);
#pragma unroll
    for (int j = 0; j < kDRows; ++j, p += kBPX) {
      const Sp<float> pn = S(sp[p + kBPX]);
      utm = dsite(dx, dy0 + j, pm, pc, pn, utm);
      pm = pc;
      pc = pn;
    }
  } else if (tid < 6 * kBX + 2 * kBDY) {
    const int k = tid - 6 * kBX;
    const int dx = k < kBDY ? 0 : kBDX - 1, dy = k % kBDY;
    const int p = (dy + 1) * kBPX + dx + 1, u = (dy + 1) * kBUX + dx + 1;
    dsite(dx, dy, S(sp[p - kBPX]), S(sp[p]), S(sp[p + kBPX]), UT(u - kBUX));
  }
  __syncthreads();

  // D^dag down a 4-row column strip per thread (64 columns x 4 strips): the
  // t-neighbours and U_t(n - t) of the strip come from registers
  constexpr int kRows = kBY / (kBT / kBX);
  const int tx = tid % kBX, ty0 = (tid / kBX) * kRows;
  const int x = x0 + tx;
  int d = (ty0 + 1) * kBDX + tx + 1, u = (ty0 + 2) * kBUX + tx + 2;
  Sp<float> tm = S(st[d - kBDX]), tc = S(st[d]);
  Cx<float> utm = UT(u - kBUX);
#pragma unroll
  for (int j = 0; j < kRows; ++j, d += kBDX, u += kBUX) {
    const Sp<float> tn = S(st[d + kBDX]);
    const float4 uu = su[u];
    const int t = t0 + ty0 + j;
    if (x < L && t < T) {
      const Sp<float> o = hop_sum<true, float>(S(st[d + 1]), S(st[d - 1]), tn, tm, {uu.x, uu.y},
                                               UX(u - 1), {uu.z, uu.w}, utm);
      const Sp<float> r = diag * tc - 0.5f * o;
      reinterpret_cast<float4*>(out)[off + x + (long long)L * t] =
          make_float4(r.a.re, r.a.im, r.b.re, r.b.im);
    }
    tm = tc;
    tc = tn;
    utm = {uu.z, uu.w};
  }
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
    const size_t smem = sizeof(float4) * (kBPX * kBPY + kBUX * kBUY + kBDX * kBDY);
    cudaError_t e = cudaFuncSetAttribute(k_ddagd_tile_big,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(SM_ERR_CUDA, "ddagd attribute: %s", cudaGetErrorString(e));
    k_ddagd_tile_big<<<c.L->ntiles_big, kBT, smem, c.s>>>(
        c.L->d_chains, c.L->d_tiles_big, (const float*)U, (const float*)in, (float*)out);
    return launched(c.st, "ddagd_tile_big");
  }
  k_ddagd_tile<R><<<c.L->ntiles, kTX * kTY, 0, c.s>>>(c.L->d_chains, c.L->d_tiles, U, in, out);
  return launched(c.st, "ddagd_tile");
}
template int launch_ddagd<float>(Ctx&, const float*, const float*, float*);
template int launch_ddagd<double>(Ctx&, const double*, const double*, double*);

}  // namespace sm
