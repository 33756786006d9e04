// tile.cuh -- the 64 x 16-tile fused D^dag D in FP32 (D in kept on chip),
// shared by sm_apply_DdagD (ddagd.cu) and the grid-wide CG (cg_tiled.cu).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace sm {

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

constexpr size_t kBigSmemBytes = sizeof(float4) * (kBPX * kBPY + kBUX * kBUY + kBDX * kBDY);

// TMA staging of an interior tile of a single-chain lattice.  The FP32
// spinor and link fields, 16 bytes per site, are described to the tensor
// memory accelerator as 2D arrays of FP64 pairs: (2 L) x T elements, so a box
// row of 68 sites is 136 elements (box sides are limited to 256).  Box
// origins use x = 2 (x0 - 2), always even: 16-byte aligned.
constexpr unsigned kTmaInBytes = 2 * kBPX * kBPY * 8;
constexpr unsigned kTmaUBytes = 2 * kBUX * kBUY * 8;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// Stages `in` and U of an interior tile by two box copies completing on
// `bar`; returns false (and records err) if they did not complete within
// `spin` polls of the barrier (kTmaSpin unless the lattice's limit was
// lowered).  The wait after a give-up, for copies still landing in this
// block's shared memory, keeps its full bound whatever `spin` is.
__device__ __forceinline__ bool tma_stage(float4* sp, float4* su, const CUtensorMap* tin,
                                          const CUtensorMap* tU, int x0, int t0,
                                          unsigned long long* bar, int* err, int spin) {
  const unsigned b = smem_u32(bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b),
                 "r"(kTmaInBytes + kTmaUBytes)
                 : "memory");
    const int cx = 2 * (x0 - 2), cy = t0 - 2;
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(sp)),
        "l"(reinterpret_cast<unsigned long long>(tin)), "r"(cx), "r"(cy), "r"(b)
        : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(su)),
        "l"(reinterpret_cast<unsigned long long>(tU)), "r"(cx), "r"(cy), "r"(b)
        : "memory");
  }
  auto poll = [&]() {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(b)
        : "memory");
    return ok;
  };
  unsigned done = 0;
  for (int i = 0; i < spin && !done; ++i) done = poll();
  if (!done) {
    if (threadIdx.x == 0 && err) atomicOr(err, 1);
    // the copies may still be landing in this block's shared memory: wait for
    // them (again bounded) before the block gives up its tile and exits
    unsigned late = 0;
    for (int i = 0; i < 16 * kTmaSpin && !late; ++i) late = poll();
  }
  return __syncthreads_and(done) != 0;
}

// out = D^dag D in on one 64 x 16 tile (tile.x = chain, tile.y = x0,
// tile.z = t0) of the batch; `sm4` is the block's dynamic shared memory
// (kBigSmemBytes).  If `norm` is not NULL it receives this thread's part of
// |D in|^2 over the tile's own sites (the D stage also computes the ring).
// With tin and tU (tensor maps of `in` and U, single-chain lattices only),
// interior tiles are staged by TMA; `err` (may be NULL) records a box copy
// that did not complete, in which case the tile is not computed.
__device__ __forceinline__ void ddagd_big_tile(float4* sm4, const ChainInfo& ci, int4 tile,
                                               const float* __restrict__ U,
                                               const float* __restrict__ in,
                                               float* __restrict__ out, float* norm,
                                               const CUtensorMap* tin = nullptr,
                                               const CUtensorMap* tU = nullptr,
                                               unsigned long long* bar = nullptr,
                                               int* err = nullptr, int spin = kTmaSpin) {

  float4* sp = sm4;                   // [kBPY][kBPX]
  float4* su = sp + kBPX * kBPY;      // [kBUY][kBUX]
  float4* st = su + kBUX * kBUY;      // [kBDY][kBDX]
  const int x0 = tile.y, t0 = tile.z, L = ci.L, T = ci.T;
  const long long off = ci.off;
  const int tid = threadIdx.x;
  const float4* in4 = reinterpret_cast<const float4*>(in) + off;
  const float4* U4 = reinterpret_cast<const float4*>(U) + off;
  const bool interior = x0 >= 2 && x0 + kBX + 2 <= L && t0 >= 2 && t0 + kBY + 2 <= T;
  if (interior && tin) {
    if (!tma_stage(sp, su, tin, tU, x0, t0, bar, err, spin)) return;
  } else if (interior) {
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
    if (norm && dx >= 1 && dx <= kBX && dy >= 1 && dy <= kBY && x0 + dx - 1 < L && t0 + dy - 1 < T)
      *norm += norm2(tv);
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

}  // namespace sm
