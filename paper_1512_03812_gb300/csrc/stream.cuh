// stream.cuh -- warp-streaming fused D^dag D in FP32 (Eq. fer_action's
// operator on large lattices), shared by sm_apply_DdagD (ddagd.cu) and the
// grid-wide CG (cg_tiled.cu).
//
// One warp owns a strip of 60 output columns and TT output rows of one chain
// and walks along it row by row.  Its window is 64 columns wide (two sites
// per lane: 2 l and 2 l + 1 of the window) and starts two columns left of the
// strip; the walk reads rows ts - 2 .. ts + TT + 1, down or up.  Each row of
// `in` and U reaches shared memory by 16-byte cp.async copies into a per-warp
// ring of kSStages rows, so a warp keeps kSStages - 1 rows in flight with no
// block barrier; from there each lane takes its two sites into registers.
// The stencil then runs on registers: t-neighbours are the rows held from the
// previous steps, x-neighbours inside a lane's pair are its own, across lanes
// one shuffle.  At each step D is computed on the row read one step earlier
// and D^dag on the row read two steps earlier.  D is valid on window columns
// 1 .. 62 and D^dag D on 2 .. 61, the strip.  Every coordinate wraps
// periodically (the antiperiodic sign is in U), so any L and T work; strips
// at the right edge are narrower and rows past T are skipped.  Global
// traffic per site is 32 bytes read (in, U) and 16 written, plus the window's
// halo re-reads (x 1.07 x 1.13 at TT = 30), which neighbouring strips running
// at the same time find in L2.
#pragma once

#include "common.cuh"

namespace sm {

constexpr int kSW = 64;          // window columns per warp
constexpr int kSOut = kSW - 4;   // output columns per warp
constexpr int kSWarps = 4;       // warps per block (all on one chain)
constexpr int kSStages = 4;      // ring depth in rows
constexpr int kSThreads = 32 * kSWarps;
constexpr int kSRing = kSStages * 2 * kSW;  // float4 per warp: `in` then U per stage

// The CG form of the walk (cg_tiled.cu): its input is the search direction
// p = r + beta p_old, formed for every window site from r and p_old; the
// strip's own sites also store p (into pnew) and take x += alpha_x p_old (the
// previous iteration's update of the iterate, by reductions the warp does not
// wait for).  The ring then holds r, U and p_old per row.
struct CgFuse {
  const float* pold;
  float* pnew;
  float* x;
  float beta, alpha_x;
};
constexpr int kSRingCG = kSStages * 3 * kSW;  // float4 per warp in the CG form

// Ring slot of window site s: pairs of slots are swapped in every second
// group of 8, so that a lane reading sites 2 l (or 2 l + 1) and the copies
// writing sites l, l + 32 both touch 32 distinct banks per quarter-warp.
__device__ __forceinline__ int sswz(int s) { return s ^ ((s >> 3) & 1); }

__device__ __forceinline__ void cp_async16s(float4* smem, const float4* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ Sp<float> f4sp(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }

__device__ __forceinline__ float4 shfl_up4(float4 v) {
  v.x = __shfl_up_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_up_sync(0xffffffffu, v.y, 1);
  v.z = __shfl_up_sync(0xffffffffu, v.z, 1);
  v.w = __shfl_up_sync(0xffffffffu, v.w, 1);
  return v;
}
__device__ __forceinline__ float4 shfl_down4(float4 v) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_down_sync(0xffffffffu, v.y, 1);
  v.z = __shfl_down_sync(0xffffffffu, v.z, 1);
  v.w = __shfl_down_sync(0xffffffffu, v.w, 1);
  return v;
}

// out = D^dag D in on the strip (xs, ts) of chain ci, TT rows; `ring` is the
// warp's kSRing float4 of shared memory.  The walk goes down the rows (t
// increasing) or, if UP, up them: vertically adjacent strips walk in opposite
// directions, so the 4 window rows they share are read by both at about the
// same time (at the start of both walks, or at the end of both) and the second
// read finds them in L2.  Returns this lane's part of |D in|^2 over the
// strip's own sites if NORM.  Call from all 32 lanes.
template <bool NORM, bool UP, bool CG = false>
__device__ __forceinline__ float ddagd_stream_walk(float4* ring, const ChainInfo& ci, int xs,
                                                   int ts, int TT, const float* __restrict__ U,
                                                   const float* __restrict__ in,
                                                   float* __restrict__ out, const CgFuse& cgf) {
  constexpr int NP = CG ? 3 : 2;  // planes per ring stage: in (or r), U, [p_old]
  const int lane = threadIdx.x & 31;
  const int L = ci.L, T = ci.T;
  const float4* in4 = reinterpret_cast<const float4*>(in) + ci.off;
  const float4* U4 = reinterpret_cast<const float4*>(U) + ci.off;
  float4* out4 = reinterpret_cast<float4*>(out) + ci.off;
  auto wrap = [](int v, int n) { v %= n; return v < 0 ? v + n : v; };
  // the two sites this lane copies (window sites lane, lane + 32) and the two
  // it computes (2 lane, 2 lane + 1)
  const int cx0 = wrap(xs - 2 + lane, L), cx1 = wrap(xs + 30 + lane, L);
  const int ncols = min(kSOut, L - xs);  // output columns of the strip
  const int s0 = 2 * lane;
  // window site s is output column xs + s - 2
  const bool out0 = s0 >= 2 && s0 - 2 < ncols, out1 = s0 >= 1 && s0 - 1 < ncols;
  const int nrows = TT + 4;
  const int trows = T - ts;  // strip rows past this are outside the lattice
  // the walk carries 2 D in (2 diag in - hop, one FMA per component) and
  // forms 4 D^dag D in the same way; the powers of two are exact, and the
  // result and |D in|^2 are scaled once at the end
  const float diag2 = (float)(2.0 * (2.0 + ci.m0));
  auto twice_d = [&](const Sp<float>& v, const Sp<float>& h) {
    return Sp<float>{{fmaf(diag2, v.a.re, -h.a.re), fmaf(diag2, v.a.im, -h.a.im)},
                     {fmaf(diag2, v.b.re, -h.b.re), fmaf(diag2, v.b.im, -h.b.im)}};
  };

  // step i reads window row i (down) or nrows - 1 - i (up); window row w is
  // lattice row ts - 2 + w
  int tload = UP ? wrap(ts + TT + 1, T) : wrap(ts - 2, T);
  int iload = 0;
  const float4* po4 = CG ? reinterpret_cast<const float4*>(cgf.pold) + ci.off : nullptr;
  auto issue = [&]() {
    if (iload < nrows) {
      float4* st = ring + (iload % kSStages) * (NP * kSW);
      const long long ro = (long long)L * tload;
      cp_async16s(st + sswz(lane), in4 + ro + cx0);
      cp_async16s(st + sswz(lane + 32), in4 + ro + cx1);
      cp_async16s(st + kSW + sswz(lane), U4 + ro + cx0);
      cp_async16s(st + kSW + sswz(lane + 32), U4 + ro + cx1);
      if (CG) {
        cp_async16s(st + 2 * kSW + sswz(lane), po4 + ro + cx0);
        cp_async16s(st + 2 * kSW + sswz(lane + 32), po4 + ro + cx1);
      }
      if (UP)
        tload = tload == 0 ? T - 1 : tload - 1;
      else
        tload = tload + 1 == T ? 0 : tload + 1;
    }
    ++iload;
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
#pragma unroll
  for (int k = 0; k < kSStages - 1; ++k) issue();

  // three-row register rings, slot = step mod 3: at step i, `cur` holds the
  // row just read, p1 the one before it in walk order, p2 the one before that.
  // Walking up, the links of row i are taken at step i (D on row i - 1 needs
  // U_t of the row below it, row i).  Walking down they are taken one step
  // later, so that slot `cur` still holds the links of row i - 3, whose U_t
  // D^dag on row i - 2 needs.
  Sp<float> in_[3][2], D_[3][2];
  float4 U_[3][2] = {};  // (Ux.re, Ux.im, Ut.re, Ut.im) of the lane's two sites
  Cx<float> uxl[3];      // U_x of the site left of 2 lane, per row
  float nrm = 0.f;
#pragma unroll 1
  for (int i0 = 0; i0 < nrows; i0 += 3) {
#pragma unroll
    for (int ph = 0; ph < 3; ++ph) {
      const int i = i0 + ph;
      if (i >= nrows) break;
      const int cur = ph, p1 = (ph + 2) % 3, p2 = (ph + 1) % 3;
      if (!UP && i >= 1) {
        // links of row i - 1, before the copy of this step reuses its stage
        const float4* sp = ring + ((i - 1) % kSStages) * (NP * kSW);
        U_[p1][0] = sp[kSW + sswz(s0)];
        U_[p1][1] = sp[kSW + sswz(s0 + 1)];
        __syncwarp();
      }
      issue();
      asm volatile("cp.async.wait_group %0;\n" ::"n"(kSStages - 1) : "memory");
      __syncwarp();
      const float4* st = ring + (i % kSStages) * (NP * kSW);
      in_[cur][0] = f4sp(st[sswz(s0)]);
      in_[cur][1] = f4sp(st[sswz(s0 + 1)]);
      if (CG) {
        // p = r + beta p_old on the window; the strip's own sites store p
        // and add alpha_x p_old to x
        const Sp<float> po0 = f4sp(st[2 * kSW + sswz(s0)]), po1 = f4sp(st[2 * kSW + sswz(s0 + 1)]);
        in_[cur][0] = in_[cur][0] + cgf.beta * po0;
        in_[cur][1] = in_[cur][1] + cgf.beta * po1;
        const int sr = (UP ? nrows - 1 - i : i) - 2;  // strip row of the row read
        if (sr >= 0 && sr < TT && sr < trows) {
          const long long ro = (long long)L * (ts + sr) + xs - 2 + s0;
          float4* pn4 = reinterpret_cast<float4*>(cgf.pnew) + ci.off;
          float4* x4 = reinterpret_cast<float4*>(cgf.x) + ci.off;
          const float ax = cgf.alpha_x;
          if (out0) {
            const Sp<float>& v = in_[cur][0];
            pn4[ro] = make_float4(v.a.re, v.a.im, v.b.re, v.b.im);
            if (ax != 0.f)
              red_add4s(x4 + ro, make_float4(ax * po0.a.re, ax * po0.a.im, ax * po0.b.re,
                                             ax * po0.b.im));
          }
          if (out1) {
            const Sp<float>& v = in_[cur][1];
            pn4[ro + 1] = make_float4(v.a.re, v.a.im, v.b.re, v.b.im);
            if (ax != 0.f)
              red_add4s(x4 + ro + 1, make_float4(ax * po1.a.re, ax * po1.a.im, ax * po1.b.re,
                                                 ax * po1.b.im));
          }
        }
      }
      if (UP) {
        U_[cur][0] = st[kSW + sswz(s0)];
        U_[cur][1] = st[kSW + sswz(s0 + 1)];
      }
      __syncwarp();
      if (i >= 2) {
        // D on row p1; its t + 1 and t - 1 neighbours are rows cur and p2
        // (down) or p2 and cur (up), and so is the link U_t(n - t)
        const int tp = UP ? p2 : cur, tm = UP ? cur : p2;
        const float4 a0 = make_float4(in_[p1][0].a.re, in_[p1][0].a.im, in_[p1][0].b.re,
                                      in_[p1][0].b.im);
        const float4 a1 = make_float4(in_[p1][1].a.re, in_[p1][1].a.im, in_[p1][1].b.re,
                                      in_[p1][1].b.im);
        const Sp<float> left = f4sp(shfl_up4(a1)), right = f4sp(shfl_down4(a0));
        const Cx<float> ux0 = {U_[p1][0].x, U_[p1][0].y}, ux1 = {U_[p1][1].x, U_[p1][1].y};
        uxl[p1] = {__shfl_up_sync(0xffffffffu, ux1.re, 1), __shfl_up_sync(0xffffffffu, ux1.im, 1)};
        const Sp<float> h0 = hop_sum<false, float>(in_[p1][1], left, in_[tp][0], in_[tm][0], ux0,
                                                   uxl[p1], {U_[p1][0].z, U_[p1][0].w},
                                                   {U_[tm][0].z, U_[tm][0].w});
        const Sp<float> h1 = hop_sum<false, float>(right, in_[p1][0], in_[tp][1], in_[tm][1], ux1,
                                                   ux0, {U_[p1][1].z, U_[p1][1].w},
                                                   {U_[tm][1].z, U_[tm][1].w});
        D_[p1][0] = twice_d(in_[p1][0], h0);
        D_[p1][1] = twice_d(in_[p1][1], h1);
        const int r = UP ? TT + 2 - i : i - 3;  // strip row of this D
        if (NORM && r >= 0 && r < TT && r < trows) {
          if (out0) nrm += norm2(D_[p1][0]);
          if (out1) nrm += norm2(D_[p1][1]);
        }
      }
      if (i >= 4) {
        // D^dag on row p2, from D on rows p2, p1 (computed this step) and cur
        // (two steps ago)
        const int tp = UP ? cur : p1, tm = UP ? p1 : cur;
        const float4 d0 = make_float4(D_[p2][0].a.re, D_[p2][0].a.im, D_[p2][0].b.re,
                                      D_[p2][0].b.im);
        const float4 d1 = make_float4(D_[p2][1].a.re, D_[p2][1].a.im, D_[p2][1].b.re,
                                      D_[p2][1].b.im);
        const Sp<float> left = f4sp(shfl_up4(d1)), right = f4sp(shfl_down4(d0));
        const Cx<float> ux0 = {U_[p2][0].x, U_[p2][0].y}, ux1 = {U_[p2][1].x, U_[p2][1].y};
        const int um = UP ? p1 : cur;  // the row below row p2
        const Cx<float> utm0 = {U_[um][0].z, U_[um][0].w};
        const Cx<float> utm1 = {U_[um][1].z, U_[um][1].w};
        const Sp<float> h0 = hop_sum<true, float>(D_[p2][1], left, D_[tp][0], D_[tm][0], ux0,
                                                  uxl[p2], {U_[p2][0].z, U_[p2][0].w}, utm0);
        const Sp<float> h1 = hop_sum<true, float>(right, D_[p2][0], D_[tp][1], D_[tm][1], ux1, ux0,
                                                  {U_[p2][1].z, U_[p2][1].w}, utm1);
        const int r = UP ? TT + 3 - i : i - 4;  // strip row of this output
        if (r < trows) {
          const long long ro = (long long)L * (ts + r) + xs - 2 + s0;
          if (out0) {
            const Sp<float> o = 0.25f * twice_d(D_[p2][0], h0);
            out4[ro] = make_float4(o.a.re, o.a.im, o.b.re, o.b.im);
          }
          if (out1) {
            const Sp<float> o = 0.25f * twice_d(D_[p2][1], h1);
            out4[ro + 1] = make_float4(o.a.re, o.a.im, o.b.re, o.b.im);
          }
        }
      }
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  return 0.25f * nrm;
}

// One entry {chain, xs, ts, dir} of the strip table: dir 1 walks down, 2 up,
// 0 is padding (returns 0).
template <bool NORM>
__device__ __forceinline__ float ddagd_stream_strip(float4* ring, const ChainInfo* chains,
                                                    int4 s, int TT, const float* __restrict__ U,
                                                    const float* __restrict__ in,
                                                    float* __restrict__ out) {
  const CgFuse none{};
  if (s.w == 1)
    return ddagd_stream_walk<NORM, false>(ring, chains[s.x], s.y, s.z, TT, U, in, out, none);
  if (s.w == 2)
    return ddagd_stream_walk<NORM, true>(ring, chains[s.x], s.y, s.z, TT, U, in, out, none);
  return 0.f;
}

// The CG form of one strip (see CgFuse): Ap = D^dag D p with p = r + beta
// p_old, returning this lane's part of |D p|^2.
__device__ __forceinline__ float ddagd_stream_strip_cg(float4* ring, const ChainInfo* chains,
                                                       int4 s, int TT, const float* __restrict__ U,
                                                       const float* __restrict__ r,
                                                       float* __restrict__ Ap, const CgFuse& f) {
  if (s.w == 1)
    return ddagd_stream_walk<true, false, true>(ring, chains[s.x], s.y, s.z, TT, U, r, Ap, f);
  if (s.w == 2)
    return ddagd_stream_walk<true, true, true>(ring, chains[s.x], s.y, s.z, TT, U, r, Ap, f);
  return 0.f;
}

}  // namespace sm
